"""Lippmann-Schwinger solves (Sec. 3.3, eq. (descretls)) at the sizes and wavenumbers the solver
is specified on: n = 512 with kappa in {10, 40, 100}, and n = 1024, 2048 with kappa = 40, for the
smooth contrast 0.5 bump(0.4) and the Fourier-smoothed disk contrast 0.5 chi^n psi (disk of
radius 0.3, Sec. 2.4), in FP64 and in mixed precision (FP32 matvecs inside FP64 refinement).

Checks, as in test_gpu_ls: the GPU solution's true residual, evaluated by the ORACLE's FP64
operator, is <= 1.05e-10; at n = 512 the solution also agrees with the oracle's tight (1e-13)
GMRES solve to 1e-8 relative L-infinity.
"""
import functools

import numpy as np
import pytest
import torch

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, ls_solve

pytestmark = pytest.mark.gpu

A3 = O.default_trunc_radius(3.0)


@functools.lru_cache(maxsize=None)
def _contrast(n, kind):
    if kind == "bump":
        return inputs.lippmann_contrast(n, "bump")
    return 0.5 * O.fs_mask(n, 3.0, "disk", (0.5, 0.5, 0.3), 0.15)


@functools.lru_cache(maxsize=None)
def _ghat(n, kappa):
    return O.ghat_full("helm", 3 * n, 3.0, A3, kappa=kappa)


@functools.lru_cache(maxsize=None)
def _tight(n, kappa, kind):
    m = _contrast(n, kind)
    f = inputs.plane_wave(n, kappa)
    x, it, rr, ok = O.gmres(f, 3 * n, _ghat(n, kappa), kappa, m, tol=1e-13, maxit=4000)
    assert ok
    return x


CASES = [(512, 10.0), (512, 40.0), (512, 100.0), (1024, 40.0), (2048, 40.0)]


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("contrast", ["bump", "fsdisk"])
@pytest.mark.parametrize("n,kappa", CASES)
def test_ls_solve_at_size(n, kappa, contrast, mode):
    m = _contrast(n, contrast)
    f = inputs.plane_wave(n, kappa)
    prec = "fp64" if mode == "fp64" else "fp32"
    plan = ConvPlan("helmholtz", n=n, period=3, precision=prec, io="c2c", kappa=kappa, compact=True)
    x, info = ls_solve(plan, torch.tensor(m, device="cuda"), torch.tensor(f, device="cuda"),
                       tol=1e-10, restart=50, refine=(mode == "mixed"))
    plan.device_status()
    assert info["status"] == "CONV_OK", info
    xg = x.cpu().numpy()
    del plan
    r = f - O.ls_apply(xg, 3 * n, _ghat(n, kappa), kappa, m)
    rr = np.linalg.norm(r) / np.linalg.norm(f)
    assert rr <= 1.05e-10, (rr, info)
    assert abs(info["rel_residual"] - rr) <= 1e-11 + 0.05 * rr, (rr, info)
    if n == 512:
        xref = _tight(n, kappa, contrast)
        assert np.max(np.abs(xg - xref)) / np.max(np.abs(xref)) <= 1e-8


def test_ls_solve_period_b_plan_at_n512():
    """The same solve on the paper's period-3 passes (not the compact grid)."""
    n, kappa = 512, 40.0
    m = _contrast(n, "fsdisk")
    f = inputs.plane_wave(n, kappa)
    plan = ConvPlan("helmholtz", n=n, period=3, precision="fp32", io="c2c", kappa=kappa)
    x, info = ls_solve(plan, torch.tensor(m, device="cuda"), torch.tensor(f, device="cuda"), tol=1e-10, refine=True)
    assert info["status"] == "CONV_OK", info
    xg = x.cpu().numpy()
    r = f - O.ls_apply(xg, 3 * n, _ghat(n, kappa), kappa, m)
    assert np.linalg.norm(r) / np.linalg.norm(f) <= 1.05e-10
    xref = _tight(n, kappa, "fsdisk")
    assert np.max(np.abs(xg - xref)) / np.max(np.abs(xref)) <= 1e-8
