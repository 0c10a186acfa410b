"""Parity of the CUDA path with the oracle at the sizes the method is specified on.

  - Fourier-smoothed convolutions (Sec. 2.4, eq. (tfs)): the disk indicator times a smooth
    factor and the square indicator, log and |x|^-1 kernels, n = 1024 ... 4096, FP64 and FP32,
    element by element against the oracle's FFT convolution with the oracle's mask.
  - The convergence of Fourier smoothing (Table 8: second order for the log kernel) on the GPU
    path alone, against the closed-form potentials of the square, up to n = 4096 in FP64, and the
    FP32 passes up to n = 8192 (where FP32 rounding, not the discretisation, sets the error).
  - The |x|^gamma kernels (Sec. 2.2) at n = 4096, batch 16, the benchmark's launch configuration.
  - A non-integer period, b = 5/2 (Sec. 2.1 uses only that n b is an integer).

Tolerances as in test_gpu_conv: 1e-12 (FP64), 2e-6 (FP32) relative L-infinity.
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

TOL = {"fp64": 1e-12, "fp32": 2e-6}
INV2PI = 1.0 / (2.0 * math.pi)
SQUARE = (0.25, 0.75, 0.25, 0.75)
DISK = (0.5, 0.5, 0.3)


def _relerr(ref, got):
    return float(np.max(np.abs(ref - got)) / np.max(np.abs(ref)))


def _kernel(name):
    if name == "log":
        return dict(kernel="log", scale=-INV2PI), ("log", dict(scale=-INV2PI))
    return dict(kernel="pow", gamma=-1.0), ("pow", dict(gamma=-1.0))


def _fs_density(n, shape):
    """(u~, geometry): the disk workload multiplies the smoothed indicator by a seeded smooth
    factor; the square workload is the bare indicator."""
    if shape == "disk":
        return inputs.smooth_extension(n), DISK
    return np.ones((n, n)), SQUARE


@pytest.mark.parametrize("n,prec,compact", [(1024, "fp64", False), (1024, "fp32", True), (2048, "fp64", True),
                                            (2048, "fp32", False), (4096, "fp64", True), (4096, "fp32", True)])
@pytest.mark.parametrize("shape,kname", [("disk", "log"), ("square", "inv")])
def test_fourier_smoothed_convolution_at_size(n, prec, compact, shape, kname):
    kw, (okind, okw) = _kernel(kname)
    plan = ConvPlan(n=n, period=3, precision=prec, io="r2r", compact=compact, **kw)
    ut, geom = _fs_density(n, shape)
    mask = plan.fs_mask("disk" if shape == "disk" else "rect", geom, 0.15)
    out = plan.apply(torch.tensor(ut, dtype=plan.real_dtype, device="cuda"), mask=mask).cpu().numpy()
    plan.device_status()
    om = O.fs_mask(n, 3.0, "disk" if shape == "disk" else "rect", geom, 0.15)
    ref = O.conv(ut * om, plan.M, O.ghat_full(okind, plan.M, 3.0, plan.a, **okw)).real
    assert _relerr(ref, out) <= TOL[prec], _relerr(ref, out)


def _square_error(plan, kname, n, sq=SQUARE):
    X1, X2 = inputs.grid(n)
    exact = (closed_forms.rect_log_potential(X1, X2, sq[0], sq[1]) if kname == "log"
             else closed_forms.rect_inv_potential(X1, X2, sq[0], sq[1]))
    mask = plan.fs_mask("rect", sq, 0.15)
    out = plan.apply(torch.ones((n, n), dtype=plan.real_dtype, device="cuda"), mask=mask).cpu().numpy()
    plan.device_status()
    return _relerr(exact, out)


@pytest.mark.parametrize("kname,sq,lo,hi", [("log", SQUARE, 1.8, 2.3), ("log", (0.3, 0.7, 0.3, 0.7), 1.8, 2.3),
                                            ("inv", SQUARE, 0.8, 1.3)])
def test_fourier_smoothing_order_on_the_gpu(kname, sq, lo, hi):
    """Least-squares order of the GPU path's FS error against the closed-form potential of the
    square, n = 256 ... 4096, FP64 on the compact grid.  Log kernel: second order (Table 8's
    square [0.3, 0.7]^2 and the [0.25, 0.75]^2 square).  |x|^-1: first order, the rate the oracle
    shows too: the smoothed indicator drops the modes |k| > n b/2, whose coefficients fall like
    1/|k| along the edges, and ghat of |x|^-1 falls like 1/|k| (log: 1/|k|^2), so the dropped
    part of the convolution is O(1/n) (log: O(1/n^2))."""
    kw, _ = _kernel(kname)
    ns = [256, 512, 1024, 2048, 4096]
    errs = []
    for n in ns:
        plan = ConvPlan(n=n, period=3, precision="fp64", io="r2r", compact=True, **kw)
        errs.append(_square_error(plan, kname, n, sq))
        del plan
    order = -np.polyfit(np.log2(ns), np.log2(errs), 1)[0]
    assert lo < order < hi, (order, errs)


def test_fourier_smoothing_fp32_to_n8192():
    """The FP32 passes on the compact grid from n = 1024 to 8192: the error against the closed-form
    potential is the FS discretisation error (second order, measured in FP64 above) plus FP32
    rounding of 2n-point transforms; both stay below 3e-6 and the error does not grow with n
    beyond the rounding."""
    kw, _ = _kernel("log")
    errs = {}
    for n in (1024, 2048, 4096, 8192):
        plan = ConvPlan(n=n, period=3, precision="fp32", io="r2r", compact=True, **kw)
        errs[n] = _square_error(plan, "log", n)
        del plan
        torch.cuda.empty_cache()
    assert max(errs.values()) < 3e-6, errs
    assert errs[8192] < 2 * errs[1024] + 1e-6, errs


@pytest.mark.parametrize("gamma", [-0.5, -1.0, -1.5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pow_kernels_at_full_size(gamma, prec):
    """n = 4096, b = 3, batch 16 (the benchmark's launch configuration, compact grid): densities 0
    and 15 of the kernel sweep against the oracle's full FFT convolution."""
    n, B = 4096, 16
    plan = ConvPlan("pow", n=n, period=3, precision=prec, io="r2r", batch_max=B, compact=True, gamma=gamma)
    u = inputs.bump_sums(n, B)
    out = plan.apply(torch.tensor(u, dtype=plan.real_dtype, device="cuda"))
    plan.device_status()
    g = O.ghat_full("pow", plan.M, 3.0, plan.a, gamma=gamma)
    picks = (0, 15) if prec == "fp64" else (15,)
    ref = O.conv(u[list(picks)], plan.M, g).real
    for j, i in enumerate(picks):
        assert _relerr(ref[j], out[i].cpu().numpy()) <= TOL[prec]


@pytest.mark.parametrize("n", [64, 256, 1024])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,io,compact", [("log", "r2r", False), ("helm", "r2c", False), ("log", "r2r", True),
                                             ("helm", "c2c", True)])
def test_period_five_halves_matches_oracle(n, prec, name, io, compact):
    """b = 5/2 (M = 2.5 n; the admissible radii sqrt 2 <= a <= 3/2 of eq. (io), default the
    midpoint): the GPU's moments on the period-5/2 grid and its passes (period-b or compact)
    against the oracle at the same b and a."""
    kw = dict(kernel="log", scale=-INV2PI) if name == "log" else dict(kernel="helmholtz", kappa=20.0)
    plan = ConvPlan(n=n, period=2.5, precision=prec, io=io, batch_max=2, compact=compact, **kw)
    assert plan.info.M == 5 * n // 2 and abs(plan.a - 0.5 * (math.sqrt(2) + 1.5)) < 1e-15
    u = inputs.bump_sums(n, 2, seed=250 + n)
    if io == "c2c":
        u = u + 0.5j * inputs.bump_sums(n, 2, seed=251 + n)
    out = plan.apply(torch.tensor(u, dtype=plan.in_dtype(), device="cuda")).cpu().numpy()
    plan.device_status()
    okind = "log" if name == "log" else "helm"
    okw = dict(scale=-INV2PI) if name == "log" else dict(kappa=20.0)
    ref = O.conv(u, plan.M, O.ghat_full(okind, plan.M, 2.5, plan.a, **okw))
    if io == "r2r":
        ref = ref.real
    for i in range(2):
        assert _relerr(ref[i], out[i]) <= TOL[prec], (i, _relerr(ref[i], out[i]))
