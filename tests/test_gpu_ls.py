"""Lippmann-Schwinger solve (Sec. 3.3, eq. (descretls)) on the GPU against the CPU oracle.

Several solutions are correct at a 1e-10 residual; what is unique is the exact solution of the
Nystrom system, which the oracle approximates with a tight (1e-13) GMRES solve.  Checks:
  - the GPU solution's true residual, evaluated by the ORACLE's FP64 operator, is <= 1.05e-10;
  - the GPU solution agrees with the oracle's tight solve to 1e-8 relative L-infinity.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, ls_solve, ls_solve_multi

pytestmark = pytest.mark.gpu


def _oracle(n, kappa, contrast):
    lp_M = 3 * n
    a = O.default_trunc_radius(3.0)
    g = O.ghat_full("helm", lp_M, 3.0, a, kappa=kappa)
    m = inputs.lippmann_contrast(n, contrast)
    f = inputs.plane_wave(n, kappa)
    x, it, rr, ok = O.gmres(f, lp_M, g, kappa, m, tol=1e-13, maxit=4000)
    assert ok
    return g, m, f, x


def _true_residual(g, M, kappa, m, f, x):
    r = f - O.ls_apply(x, M, g, kappa, m)
    return np.linalg.norm(r) / np.linalg.norm(f)


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("n,kappa,contrast", [(32, 10.0, "bump"), (64, 10.0, "disk"), (64, 40.0, "bump")])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ls_solve_matches_oracle(n, kappa, contrast, mode, compact):
    g, m, f, xref = _oracle(n, kappa, contrast)
    prec = "fp64" if mode == "fp64" else "fp32"
    plan = ConvPlan("helmholtz", n=n, period=3, precision=prec, io="c2c", kappa=kappa, compact=compact)
    x, info = ls_solve(plan, torch.tensor(m, device="cuda"), torch.tensor(f, device="cuda"),
                       tol=1e-10, restart=50, refine=(mode == "mixed"))
    assert info["status"] == "CONV_OK", info
    xg = x.cpu().numpy()
    rr = _true_residual(g, plan.M, kappa, m, f, xg)
    assert rr <= 1.05e-10, (rr, info)
    assert np.max(np.abs(xg - xref)) / np.max(np.abs(xref)) <= 1e-8
    assert info["rel_residual"] <= 1.05e-10


def test_ls_solve_reports_nonconvergence_and_repeats_bitwise():
    n, kappa = 32, 20.0
    _, m, f, _ = _oracle(n, kappa, "bump")
    plan = ConvPlan("helmholtz", n=n, period=3, precision="fp64", io="c2c", kappa=kappa)
    mt, ft = torch.tensor(m, device="cuda"), torch.tensor(f, device="cuda")
    x, info = ls_solve(plan, mt, ft, tol=1e-14, max_iters=3, restart=2)
    assert info["status"] == "CONV_ENOTCONVERGED" and info["iters"] == 3
    x1, _ = ls_solve(plan, mt, ft, tol=1e-10)
    x2, _ = ls_solve(plan, mt, ft, tol=1e-10)
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ls_solve_multi_matches_oracle_per_right_hand_side(mode):
    """Three incident directions on one scatterer, one of them 1000 times larger, as one stacked
    solve: every system's true residual by the ORACLE's operator is <= 1.05e-10 (the per-system
    bound the unit-norm stacking gives), its reported residual agrees, and each solution matches
    its own single-right-hand-side solve to 1e-8."""
    n, kappa = 48, 10.0
    M = 3 * n
    g = O.ghat_full("helm", M, 3.0, O.default_trunc_radius(3.0), kappa=kappa)
    m = inputs.lippmann_contrast(n, "bump")
    F = np.stack([inputs.plane_wave(n, kappa, a) for a in (0.0, 0.7, 2.1)])
    F[1] *= 1000.0
    prec = "fp64" if mode == "fp64" else "fp32"
    plan = ConvPlan("helmholtz", n=n, period=3, precision=prec, io="c2c", kappa=kappa)
    mt = torch.tensor(m, device="cuda")
    X, infos = ls_solve_multi(plan, mt, torch.tensor(F, device="cuda"), tol=1e-10, refine=(mode == "mixed"))
    Xg = X.cpu().numpy()
    for s in range(3):
        assert infos[s]["status"] == "CONV_OK", infos
        rr = _true_residual(g, M, kappa, m, F[s], Xg[s])
        assert rr <= 1.05e-10, (s, rr, infos[s])
        assert abs(infos[s]["rel_residual"] - rr) <= 1e-11 + 0.05 * rr, (rr, infos[s])
        x1, _ = ls_solve(plan, mt, torch.tensor(F[s], device="cuda"), tol=1e-10, refine=(mode == "mixed"))
        x1 = x1.cpu().numpy()
        assert np.max(np.abs(Xg[s] - x1)) / np.max(np.abs(x1)) <= 1e-8
    # an initial guess near the solution: fewer iterations, same bound
    X0 = torch.tensor(Xg * (1 + 1e-6), device="cuda")
    X2, infos2 = ls_solve_multi(plan, mt, torch.tensor(F, device="cuda"), X=X0, tol=1e-10, refine=(mode == "mixed"))
    X2g = X2.cpu().numpy()
    for s in range(3):
        assert _true_residual(g, M, kappa, m, F[s], X2g[s]) <= 1.05e-10
    assert infos2[0]["iters"] < infos[0]["iters"]


def test_ls_solve_multi_with_one_right_hand_side_is_ls_solve():
    """count = 1 runs the plain solve: bitwise the same solution and residual."""
    n, kappa = 32, 10.0
    _, m, f, _ = _oracle(n, kappa, "bump")
    plan = ConvPlan("helmholtz", n=n, period=3, precision="fp32", io="c2c", kappa=kappa)
    mt, ft = torch.tensor(m, device="cuda"), torch.tensor(f, device="cuda")
    x1, i1 = ls_solve(plan, mt, ft, refine=True)
    X, infos = ls_solve_multi(plan, mt, ft[None].contiguous(), refine=True)
    assert torch.equal(X[0], x1)
    assert infos[0]["rel_residual"] == i1["rel_residual"] and infos[0]["iters"] == i1["iters"]
