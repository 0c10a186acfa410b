"""conv_apply_kernels: one batch of densities, each convolved with its own plan's kernel, in one
launch per pass on a shape plan; every result is bitwise its own conv_apply (the same kernels and
arithmetic, only the multiplier table chosen per density)."""
import math

import numpy as np
import pytest
import torch

from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300._native import ConvError
from paper_2107_03958_gb300.api import ConvPlan, apply_kernels

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("io,n", [("r2r", 256), ("r2c", 128), ("c2c", 96), ("r2r", 45)])
def test_mixed_kernel_batch_equals_separate_applies(io, n, prec, compact):
    if io == "r2r":
        specs = [("log", dict(scale=-1 / (2 * math.pi))), ("pow", dict(gamma=-0.5)), ("pow", dict(gamma=-1.0)),
                 ("pow", dict(gamma=-1.5)), ("log", dict(scale=2.0))]
    else:
        specs = [("helmholtz", dict(kappa=k)) for k in (5.0, 20.0, 33.3, 60.0)]
    period = 4 if n == 45 else 3
    plans = [ConvPlan(k, n=n, period=period, precision=prec, io=io, batch_max=8, compact=compact, **kw)
             for k, kw in specs]
    B = 7
    per = [plans[i % len(plans)] for i in range(B)]
    u = inputs.bump_sums(n, B, seed=71)
    if io == "c2c":
        u = u + 0.25j * inputs.bump_sums(n, B, seed=72)
    ut = torch.tensor(u, device="cuda").to(plans[0].in_dtype())
    mask = torch.tensor(np.random.default_rng(3).uniform(0.5, 1, (n, n)), dtype=plans[0].real_dtype, device="cuda")
    out = apply_kernels(plans[2], per, ut, mask=mask)
    torch.cuda.synchronize()
    for i in range(B):
        alone = per[i].apply(ut[i].contiguous(), mask=mask)
        assert torch.equal(alone, out[i]), i
    for p in plans:
        p.device_status()


def test_mixed_kernel_batch_rejects_other_shapes():
    a = ConvPlan("log", n=64, period=3, precision="fp32", io="r2r", batch_max=4)
    b = ConvPlan("log", n=64, period=3, precision="fp64", io="r2r", batch_max=4)
    c = ConvPlan("log", n=32, period=3, precision="fp32", io="r2r", batch_max=4)
    d = ConvPlan("log", n=64, period=3, precision="fp32", io="r2r", batch_max=4, compact=True)
    u = torch.zeros(2, 64, 64, dtype=torch.float32, device="cuda")
    for other in (b, c, d):
        with pytest.raises(ConvError, match="EINVAL"):
            apply_kernels(a, [a, other], u)
