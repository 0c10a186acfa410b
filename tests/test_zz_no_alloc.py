"""conv_apply_noalloc: the convolution run with the library's fixed device scratch array instead
of allocated workspace, for callers that cannot allocate device memory when they convolve (a
device-memory budget that forbids new allocations, a real-time loop, a host framework that owns
all device memory).

Called through the C ABI; its output must equal conv_apply's with a caller-supplied workspace
(same kernels, same arithmetic) on two calls in a row with different inputs, so a stale scratch
array would show.  Covered: every io mode (R2R, the split R2C layout of a complex multiplier with
an odd h n, C2C), a mask, a batch above the plan's batch_max that still fits the array, and the
rejection of misaligned arrays before any launch.  The file is named to be collected last.
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

SCRATCH = 32 << 20
EINVAL = 1


def _noalloc_raw(plan, u_ptr, mask_ptr, out_ptr, batch):
    lib = N.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.conv_apply_noalloc(plan.handle, ctypes.c_void_p(u_ptr),
                                  ctypes.c_void_p(mask_ptr) if mask_ptr else None,
                                  ctypes.c_void_p(out_ptr), int(batch), st)


def _noalloc(plan, u, out, mask=None):
    return _noalloc_raw(plan, u.data_ptr(), mask.data_ptr() if mask is not None else 0, out.data_ptr(),
                        u.shape[0] if u.dim() == 3 else 1)


def _density(plan, B, seed):
    u = inputs.bump_sums(plan.n, B, seed=seed)
    if plan.io == "c2c":
        u = u * (1.0 + 0.5j)
    return torch.tensor(u, device="cuda").to(plan.in_dtype())


CASES = [
    # (precision, io, kernel, n, period, batch_max, batch, masked, tolerance)
    ("fp64", "r2r", "log", 256, 3, 3, 3, False, 1e-12),
    ("fp32", "r2r", "log", 256, 3, 3, 3, False, 2e-6),
    ("fp64", "r2r", "log", 128, 3, 1, 4, True, 1e-12),       # batch above batch_max, masked
    ("fp64", "r2c", "helmholtz", 27, 4, 2, 2, False, 1e-12),  # split R2C, h n = 55 * 27 odd
    ("fp32", "r2c", "helmholtz", 256, 3, 2, 2, True, 2e-6),
    ("fp64", "c2c", "helmholtz", 128, 3, 2, 2, False, 1e-12),
    ("fp32", "c2c", "helmholtz", 128, 3, 1, 3, True, 2e-6),
]


@pytest.mark.parametrize("prec,io,kernel,n,period,bmax,B,masked,tol", CASES)
def test_noalloc_matches_conv_apply_twice(prec, io, kernel, n, period, bmax, B, masked, tol):
    plan = ConvPlan(kernel, n=n, period=period, precision=prec, io=io, batch_max=bmax,
                    kappa=20.0 if kernel == "helmholtz" else 0.0, scale=-1.0 / (2 * math.pi))
    if io == "r2c":
        assert plan.info.r2c_split == 1
    need = plan.workspace_bytes(B)
    assert need <= SCRATCH
    ws = torch.empty(need // 8 + 2, dtype=torch.float64, device="cuda")
    mask = plan.fs_mask("disk", (0.5, 0.5, 0.3)) if masked else None
    for seed in (1, 2):
        u = _density(plan, B, seed)
        ref = plan.apply(u, mask=mask, workspace=ws)
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(plan, u, out, mask) == 0, N.load().conv_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) <= tol * np.max(np.abs(r))


def test_noalloc_rejects_oversized_work():
    n = 1024
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", batch_max=1)
    assert plan.workspace_bytes(4) > SCRATCH
    u = torch.zeros(4, n, n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _noalloc(plan, u, out) == EINVAL
    msg = N.load().conv_last_error().decode()
    assert str(SCRATCH) in msg


@pytest.mark.parametrize("which", ["u", "out", "mask"])
def test_noalloc_rejects_misaligned_arrays(which):
    """A pointer off its element alignment is turned away by the host-side checks, as conv_apply
    turns it away, before any kernel is launched."""
    n = 64
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", batch_max=1)
    u = torch.zeros(n * n + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(n * n + 1, dtype=torch.float64, device="cuda")
    mask = torch.ones(n * n + 1, dtype=torch.float64, device="cuda")
    ptr = {"u": u.data_ptr(), "out": out.data_ptr(), "mask": mask.data_ptr()}
    ptr[which] += 4
    assert _noalloc_raw(plan, ptr["u"], ptr["mask"], ptr["out"], 1) == EINVAL
    assert "aligned" in N.load().conv_last_error().decode()
    torch.cuda.synchronize()
    assert torch.all(out == 0)
