"""Moments ghat(k) by high-precision quadrature of their definition (mpmath).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  This is the plain definition of eq. (ghat),
Sec. 2.2, for a radial kernel:

    ghat(k) = 2 pi int_0^a g(rho) J0(s rho) rho d rho,   s = 2 pi |k| / b,

integrated with mpmath at 20 significant digits on subintervals of half an oscillation of
J0(s rho) (rho_j = (j - 1/4) pi / s), so that each piece is smooth: tanh-sinh on the first piece
(after rho = r1 t^2, which removes the kernel's singularity at 0), adaptive Gauss-Legendre on the
others.  It uses no
closed form, series or asymptotic expansion of the moments.  It serves only to write stored
reference values (tests/golden/make_ghat_quadrature.py); nothing imports it at test time.
"""
import math

import mpmath as mp


def _g(kind, gamma, kappa):
    if kind == "log":
        return lambda r: mp.log(r)
    if kind == "pow":
        return lambda r: r ** gamma
    if kind == "helm":
        return lambda r: (1j / 4) * mp.hankel1(0, kappa * r)
    if kind == "yukawa":
        return lambda r: mp.besselk(0, kappa * r) / (2 * mp.pi)
    raise ValueError(kind)


def ghat_quadrature(kind, kmag, b, a, gamma=0.0, kappa=0.0, dps=20):
    """2 pi int_0^a g(rho) J0(2 pi |k| rho / b) rho d rho for g = log|x|, |x|^gamma,
    (i/4) H0^(1)(kappa |x|) or K0(kappa |x|)/(2 pi) (unscaled)."""
    mp.mp.dps = dps
    g = _g(kind, gamma, kappa)
    s = 2 * mp.pi * mp.mpf(kmag) / b
    a = mp.mpf(a)
    f = lambda r: g(r) * mp.besselj(0, s * r) * r
    pts = [mp.mpf(0)]
    if kmag > 0:
        j = 1
        while True:
            r = (j - mp.mpf(1) / 4) * mp.pi / s
            if r >= a:
                break
            pts.append(r)
            j += 1
    pts.append(a)
    # the first piece carries the kernel's singularity at rho = 0: substitute rho = r1 t^2
    r1 = pts[1]
    head = mp.quad(lambda t: f(r1 * t * t) * 2 * r1 * t, [0, 1])
    tail = mp.mpf(0)
    for lo, hi in zip(pts[1:-1], pts[2:]):
        tail += mp.quad(f, [lo, hi], method="gauss-legendre")
    v = 2 * mp.pi * (head + tail)
    return complex(v)
