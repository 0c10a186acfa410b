"""Closed-form potentials of indicator densities, used as exact references in the tests.

Each is pinned in tests/test_oracle_pins.py by brute-force 2-D quadrature of its definition.
"""
import math

import numpy as np


def rect_log_potential(X1, X2, s0, s1, t0=None, t1=None):
    """-(1/2pi) int_{[s0,s1] x [t0,t1]} log|x-y| dy (t0, t1 default to s0, s1), from the
    antiderivative P(X,Y) = 1/2 [XY(log(X^2+Y^2) - 3) + X^2 atan(Y/X) + Y^2 atan(X/Y)] of
    log|(X, Y)| summed over the four corners."""
    t0 = s0 if t0 is None else t0
    t1 = s1 if t1 is None else t1

    def P(X, Y):
        r2 = X * X + Y * Y
        L = np.log(np.where(r2 > 0, r2, 1.0))
        A = np.where(X != 0, X * X * np.arctan(Y / np.where(X != 0, X, 1)), 0.0)
        B = np.where(Y != 0, Y * Y * np.arctan(X / np.where(Y != 0, Y, 1)), 0.0)
        return 0.5 * (X * Y * (L - 3) + A + B)
    v = P(X1 - s0, X2 - t0) - P(X1 - s1, X2 - t0) - P(X1 - s0, X2 - t1) + P(X1 - s1, X2 - t1)
    return -v / (2 * math.pi)


def rect_inv_potential(X1, X2, s0, s1, t0=None, t1=None):
    """int_{[s0,s1] x [t0,t1]} |x-y|^-1 dy from the antiderivative
    Q(X,Y) = X asinh(Y/|X|) + Y asinh(X/|Y|) of 1/|(X, Y)| (d^2 Q/dX dY = 1/r for every sign of
    X and Y) summed over the four corners."""
    t0 = s0 if t0 is None else t0
    t1 = s1 if t1 is None else t1

    def Q(X, Y):
        A = np.where(X != 0, X * np.arcsinh(Y / np.where(X != 0, np.abs(X), 1)), 0.0)
        B = np.where(Y != 0, Y * np.arcsinh(X / np.where(Y != 0, np.abs(Y), 1)), 0.0)
        return A + B
    return Q(X1 - s0, X2 - t0) - Q(X1 - s1, X2 - t0) - Q(X1 - s0, X2 - t1) + Q(X1 - s1, X2 - t1)


def mie_disc_field(n, kappa, mu, R, centre=(0.5, 0.5), stride=1):
    """Total field u on the grid x_j = j/n (every stride-th node per axis) for the plane wave exp(i kappa x1) scattered by the
    homogeneous disc |x - centre| < R of refractive index mu (Delta u + kappa^2 mu u = 0 inside,
    Delta u + kappa^2 u = 0 outside, radiating scattered field): the separation-of-variables
    (Mie) series.  With exp(i kappa x1) = exp(i kappa c1) sum_m i^m J_m(kappa r) e^{i m theta},
    u = sum_m A_m J_m(k2 r) e^{i m theta} inside (k2 = kappa sqrt(mu)) and
    u = sum_m (i^m e^{i kappa c1} J_m(kappa r) + B_m H_m(kappa r)) e^{i m theta} outside, with A_m,
    B_m from the continuity of u and du/dr at r = R."""
    from scipy.special import hankel1, h1vp, jv, jvp
    x = np.arange(0, n, stride, dtype=np.float64) / n
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    dx, dy = X1 - centre[0], X2 - centre[1]
    r, th = np.hypot(dx, dy), np.arctan2(dy, dx)
    k2 = kappa * math.sqrt(mu)
    mmax = int(k2 * R + kappa * math.sqrt(2.0)) + 40
    inside = r < R
    u = np.zeros(X1.shape, dtype=np.complex128)
    phase = np.exp(1j * kappa * centre[0])
    for m in range(-mmax, mmax + 1):
        c = (1j ** m) * phase
        A = np.array([[jv(m, k2 * R), -hankel1(m, kappa * R)],
                      [k2 * jvp(m, k2 * R), -kappa * h1vp(m, kappa * R)]])
        am, bm = np.linalg.solve(A, np.array([c * jv(m, kappa * R), c * kappa * jvp(m, kappa * R)]))
        e = np.exp(1j * m * th)
        u += np.where(inside, am * jv(m, k2 * r), c * jv(m, kappa * r) + bm * hankel1(m, kappa * r)) * e
    return u
