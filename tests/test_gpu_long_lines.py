"""Transform lines longer than one CTA holds (the pass path's four-step FP64 line pipeline).

  - forced at small n (WSCONV_LONG_LINES=1, and WSCONV_LINE_SPLIT=1 so that every line really
    splits four-step): element-by-element parity with the oracle for R2R, R2C and C2C, a mask and
    the axpby form, FP64 and FP32 plans, period-3 and compact grids;
  - n = 8192 in FP64 on the compact grid (L = 16384): the log potential of the Laplacian of
    Table 7's Gaussian sum is minus that sum;
  - config 3's Fourier-smoothed square at n = 8192, FP64 on both grids and FP32 on the period-3
    grid (L = 24576): error against the square's closed-form log potential.
"""
import math

import closed_forms
import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan

pytestmark = pytest.mark.gpu

INV2PI = 1.0 / (2.0 * math.pi)


def _relerr(ref, got):
    return float(np.max(np.abs(ref - got)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("n,kernel,io", [(64, "log", "r2r"), (96, "helmholtz", "r2c"), (64, "helmholtz", "c2c"),
                                         (128, "pow", "r2r")])
def test_forced_long_lines_match_oracle(n, kernel, io, prec, tol, compact, monkeypatch):
    monkeypatch.setenv("WSCONV_LONG_LINES", "1")
    monkeypatch.setenv("WSCONV_LINE_SPLIT", "1")
    kw = dict(kappa=20.0) if kernel == "helmholtz" else (dict(gamma=-1.0) if kernel == "pow" else dict(scale=-INV2PI))
    B = 2
    plan = ConvPlan(kernel, n=n, period=3, precision=prec, io=io, batch_max=B, compact=compact, **kw)
    assert plan.info.long_lines == 1
    rng = np.random.default_rng(n)
    u = inputs.bump_sums(n, B, seed=n + 3)
    if io == "c2c":
        u = u + 0.5j * inputs.bump_sums(n, B, seed=n + 4)
    m = rng.uniform(0.5, 1.0, (n, n))
    alpha, beta = (2.0 - 1.0j, 0.5) if io != "r2r" else (2.0, 0.5)
    ut = torch.tensor(u, device="cuda").to(plan.in_dtype())
    out = plan.apply(ut, mask=torch.tensor(m, dtype=plan.real_dtype, device="cuda"), alpha=alpha, beta=beta)
    plan.device_status()
    okind = {"log": "log", "pow": "pow", "helmholtz": "helm"}[kernel]
    ref = beta * u + alpha * O.conv(u * m, plan.M, O.ghat_full(okind, plan.M, 3.0, plan.a, **kw))
    if io == "r2r":
        ref = ref.real
    got = out.cpu().numpy()
    for i in range(B):
        assert _relerr(ref[i], got[i]) <= tol, (i, _relerr(ref[i], got[i]))


def test_n8192_fp64_compact_matches_the_analytic_potential():
    n = 8192
    centres = [(0.6, 0.6), (0.5, 0.5), (0.35, 0.6)]
    f = inputs.gaussian_sum_laplacian(n, 250.0, centres)
    ex = -inputs.gaussian_sum(n, 250.0, centres)
    plan = ConvPlan("log", n=n, period=3, precision="fp64", io="r2r", compact=True, scale=-INV2PI)
    assert plan.info.long_lines == 1 and plan.info.transform_len == 16384
    out = plan.apply(torch.tensor(f, device="cuda")).cpu().numpy()
    plan.device_status()
    err = _relerr(ex, out)
    assert err <= 1e-11, err


@pytest.mark.parametrize("prec,compact,tol", [("fp64", True, 2e-8), ("fp64", False, 2e-8), ("fp32", False, 2e-6)])
def test_fourier_smoothed_square_at_n8192(prec, compact, tol):
    """Config 3's largest grid: the smoothed indicator of [0.25, 0.75]^2 (log kernel) against the
    closed-form potential; the FS error there is of order 1e-9 (second order from Table 8's
    1.3e-6 at n = 256)."""
    n = 8192
    plan = ConvPlan("log", n=n, period=3, precision=prec, io="r2r", compact=compact, scale=-INV2PI)
    assert plan.info.long_lines == (1 if (prec == "fp64" or not compact) else 0)
    mask = plan.fs_mask("rect", (0.25, 0.75, 0.25, 0.75), 0.15)
    out = plan.apply(torch.ones((n, n), dtype=plan.real_dtype, device="cuda"), mask=mask).cpu().numpy()
    plan.device_status()
    X1, X2 = inputs.grid(n)
    exact = closed_forms.rect_log_potential(X1, X2, 0.25, 0.75)
    err = _relerr(exact, out)
    assert err <= tol, err
