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
