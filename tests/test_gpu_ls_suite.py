"""The paper's scattering examples (Sec. 3.3, Tables 10-13) through the GPU solver.

  - parity: for each contrast (smooth-mu disc, filter disc, Luneburg lens, the Fourier-smoothed
    disc with m = -1) the GPU solution's true residual, evaluated by the ORACLE's FP64 operator,
    is <= 1.05e-10 in FP64 and in mixed precision, at n = 128 with the sizes kappa a of the tables;
  - convergence: the GPU path's errors against its own n = 1024 solution reproduce Table 10
    (kappa a = 50) and Table 12 (kappa a = 40 pi) within a factor 2 where their printed errors
    sit well above round-off, and against the Mie series Table 13's Fourier-smoothed column to
    n = 1024 (second order) with the unsmoothed errors far above it.
Readings as in tests/test_oracle_ls_suite.py.
"""
import math

import closed_forms
import numpy as np
import pytest
import torch
from conftest import load_golden

import oracle as O
from paper_2107_03958_gb300 import inputs
from paper_2107_03958_gb300.api import ConvPlan, ls_solve

pytestmark = pytest.mark.gpu

A3 = O.default_trunc_radius(3.0)
R13 = 0.3
K13 = 40.0 / (2 * R13)


def _fs_disc(n):
    return -O.fs_mask(n, 3.0, "disk", (0.5, 0.5, R13))


CASES = {
    "smooth-disc-1": (1.0 / 0.9, inputs.smooth_disc_contrast, 50),
    "smooth-disc-50": (50.0 / 0.9, inputs.smooth_disc_contrast, 300),
    "filter-disc-2pi": (2 * math.pi, inputs.filter_disc_contrast, 50),
    "filter-disc-40pi": (40 * math.pi, inputs.filter_disc_contrast, 100),
    "luneburg-2pi": (2 * math.pi / 0.9, inputs.luneburg_contrast, 50),
    "luneburg-40pi": (40 * math.pi / 0.9, inputs.luneburg_contrast, 100),
    "fs-disc-40": (K13, _fs_disc, 600),
}


def _gpu_solve(n, kappa, m, restart, mode="fp64", compact=True, tol=1e-10, max_iters=20000):
    prec = "fp64" if mode == "fp64" else "fp32"
    plan = ConvPlan("helmholtz", n=n, period=3, precision=prec, io="c2c", kappa=kappa, compact=compact)
    x, info = ls_solve(plan, torch.tensor(m, device="cuda"), torch.tensor(inputs.plane_wave(n, kappa), device="cuda"),
                       tol=tol, restart=restart, max_iters=max_iters, refine=(mode == "mixed"))
    plan.device_status()
    assert info["status"] == "CONV_OK", info
    return x.cpu().numpy(), info


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_ls_suite_parity(case, mode):
    kappa, contrast, restart = CASES[case]
    n = 128
    m = contrast(n)
    x, info = _gpu_solve(n, kappa, m, restart, mode)
    f = inputs.plane_wave(n, kappa)
    r = f - O.ls_apply(x, 3 * n, O.ghat_full("helm", 3 * n, 3.0, A3, kappa=kappa), kappa, m)
    rr = np.linalg.norm(r) / np.linalg.norm(f)
    assert rr <= 1.05e-10, (rr, info)


def _gpu_self_errors(kappa, contrast, restart, ns, nref):
    ref, _ = _gpu_solve(nref, kappa, contrast(nref), restart, tol=1e-12)
    out = []
    for n in ns:
        x, _ = _gpu_solve(n, kappa, contrast(n), restart, tol=1e-12)
        out.append(O.rel_err(ref[::nref // n, ::nref // n], x))
    return np.array(out)


def test_table10_kappa_a_50_on_the_gpu():
    tab = load_golden("table10_ls_smooth_disc.txt")
    rows = tab[(tab[:, 0] >= 64) & (tab[:, 0] <= 256)]
    errs = _gpu_self_errors(50.0 / 0.9, inputs.smooth_disc_contrast, 300, rows[:, 0].astype(int), 1024)
    ratio = errs / rows[:, 2]
    assert np.all((ratio > 0.5) & (ratio < 2.0)), (errs, ratio)


def test_table12_kappa_a_40pi_on_the_gpu():
    tab = load_golden("table12_ls_luneburg.txt")
    rows = tab[(tab[:, 0] >= 128) & (tab[:, 0] <= 512)]
    errs = _gpu_self_errors(40 * math.pi / 0.9, inputs.luneburg_contrast, 100, rows[:, 0].astype(int), 2048)
    ratio = errs / rows[:, 2]
    assert np.all((ratio > 0.4) & (ratio < 2.5)), (errs, ratio)


def test_table13_on_the_gpu():
    """Fourier-smoothed disc (m = -1) against the Mie series, n = 128 ... 1024 (compared on a
    256 x 256 subgrid of the nodes beyond n = 256): the errors within a factor 4 below to 2 above
    the printed FS column (the disc's size is a reading) and at least second order at the top;
    the unsmoothed contrast's errors at least 10 times larger."""
    tab = load_golden("table13_ls_fs_disc.txt")
    fs = {}
    for n in (128, 256, 512, 1024):
        st = max(1, n // 256)  # the series on a 256 x 256 subgrid of the nodes
        exact = closed_forms.mie_disc_field(n, K13, 2.0, R13, stride=st)
        x, _ = _gpu_solve(n, K13, _fs_disc(n), 600)
        fs[n] = O.rel_err(exact, x[::st, ::st])
        printed = tab[tab[:, 0] == n][0, 2]
        assert 0.25 < fs[n] / printed < 2.0, (n, fs[n], printed)
    assert 1.7 < math.log2(fs[512] / fs[1024]) < 3.0, fs
    n = 1024
    x, _ = _gpu_solve(n, K13, -inputs.indicator_disk(n, (0.5, 0.5), R13), 600)
    wfs = O.rel_err(closed_forms.mie_disc_field(n, K13, 2.0, R13, stride=4), x[::4, ::4])
    assert wfs > 10 * fs[n], (wfs, fs[n])
