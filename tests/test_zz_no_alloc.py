"""conv_apply_noalloc: the convolution run with the library's fixed device scratch array instead
of allocated workspace, for callers that cannot allocate device memory when they convolve.

Called through the C ABI; its output must equal conv_apply's (same kernels, same arithmetic) on
two calls in a row with different inputs, so a stale scratch array would show.  The file is named
to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2107_03958_gb300 import _native as N
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan

pytestmark = pytest.mark.gpu


def _noalloc(plan, u, out):
    lib = N.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.conv_apply_noalloc(plan.handle, ctypes.c_void_p(u.data_ptr()), None,
                                  ctypes.c_void_p(out.data_ptr()), u.shape[0] if u.dim() == 3 else 1, st)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_noalloc_matches_conv_apply_twice(prec, tol):
    n, B = 256, 3
    plan = ConvPlan("log", n=n, period=3, precision=prec, io="r2r", batch_max=B,
                    scale=-1.0 / (2 * math.pi))
    assert plan.workspace_bytes(B) <= 32 << 20
    for seed in (1, 2):
        u = torch.tensor(inputs.bump_sums(n, B, seed=seed), dtype=plan.real_dtype, device="cuda")
        ref = plan.apply(u)
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(plan, u, out) == 0, N.load().conv_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.max(np.abs(o - r)) <= tol * np.max(np.abs(r))


def test_noalloc_rejects_oversized_work():
    n = 1024
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", batch_max=1)
    assert plan.workspace_bytes(4) > 32 << 20
    u = torch.zeros(4, n, n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _noalloc(plan, u, out) == 1  # CONV_EINVAL
    assert "32" in N.load().conv_last_error().decode() or "scratch" in N.load().conv_last_error().decode()
