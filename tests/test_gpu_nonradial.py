"""The non-radial kernel g(x) = -x1/(2 pi |x|^2) of Sec. 3.1 on the GPU: its odd multiplier
i sgn(k1) T(|k1|, |k2|) against the oracle's table, the convolution element by element against the
oracle, and Table 6 from the GPU path."""
import math

import numpy as np
import pytest
import torch
from conftest import load_golden

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300._native import ConvError
from paper_2107_03958_gb300.api import ConvPlan

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def test_table_matches_oracle():
    n = 64
    plan = ConvPlan("dx1log", n=n, period=3, precision="fp64", io="r2r")
    T = plan.ghat_quadrant()
    full = O.ghat_full("dx1log", plan.M, 3.0, plan.a)
    h = plan.M // 2
    ref = full[:h, :h + 1].imag.T  # k1 = q1 < M/2 (positive), k2 = q2 <= M/2: [k2][k1]
    assert np.max(np.abs(T[:, :h] - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,period,a", [(32, 3, 0.0), (45, 4, 0.0), (64, 3, 0.0), (128, 3, 0.0), (64, 2, 0.9)])
def test_conv_matches_oracle(n, period, a, prec):
    B = 2
    plan = ConvPlan("dx1log", n=n, period=period, trunc_a=a, precision=prec, io="r2r", batch_max=B, scale=1.5)
    u = inputs.bump_sums(n, B, seed=600 + n)
    m = np.random.default_rng(n).uniform(0.5, 1.0, (n, n))
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda"),
                     mask=torch.tensor(m, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
    plan.device_status()
    ref = O.conv(u * m, plan.M, O.ghat_full("dx1log", plan.M, plan.b, plan.a, scale=1.5))
    assert np.max(np.abs(ref.imag)) <= 1e-13 * np.max(np.abs(ref.real))
    for i in range(B):
        e = float(np.max(np.abs(out[i] - ref[i].real)) / np.max(np.abs(ref[i].real)))
        assert e <= TOL[prec], (i, e)


def test_table6_on_the_gpu():
    tab = load_golden("table6_nonradial.txt")
    for row in tab[(tab[:, 0] >= 16) & (tab[:, 0] <= 256)]:
        n = int(row[0])
        plan = ConvPlan("dx1log", n=n, period=3, precision="fp64", io="r2r")
        X1, X2 = inputs.grid(n)
        P1, P2 = X1 * (1 - X1), X2 * (1 - X2)
        cases = [(inputs.polynomial_laplacian(n, m), m * (2 * X1 - 1) * P1 ** (m - 1) * P2 ** m, row[m - 2])
                 for m in (4, 5, 6)]
        if n <= 64:
            r2 = (X1 - 0.5) ** 2 + (X2 - 0.5) ** 2
            cases.append((inputs.gaussian_sum_laplacian(n, 250.0, [(0.5, 0.5)]),
                          500.0 * (X1 - 0.5) * np.exp(-250.0 * r2), row[1]))
        for u, ex, printed in cases:
            out = plan.apply(torch.tensor(u, device="cuda")).cpu().numpy()
            e = O.rel_err(ex, out)
            if printed > 1e-15:
                assert 0.5 < e / printed < 2.0, (n, e, printed)
            else:
                assert e < 2e-15, (n, e)


def test_non_radial_kernel_outside_its_domain_is_refused():
    for kw in (dict(io="r2c"), dict(io="c2c"), dict(io="r2r", compact=True), dict(io="r2r", moments="quadrature")):
        with pytest.raises(ConvError, match="EUNSUPPORTED"):
            ConvPlan("dx1log", n=32, period=3, **kw)
