"""Seeded synthetic inputs for the convolution and Lippmann-Schwinger workloads.

This module builds densities, contrasts and incident fields on the grid x_j = j/n of D = [0,1]^2
(first array index <-> x1).  It contains none of the method's arithmetic: the CUDA path and the
CPU oracle both take their inputs from here.

Seeds follow one rule for every workload: seed = 10**6 * workload + 10**3 * log2(n) + item.
"""
import math

import numpy as np

# workload ids used in seeds
W_POISSON_BUMP = 1      # single C-infinity bump, log kernel, n = 64, b = 2
W_KERNEL_SWEEP = 2      # sums of 1-8 bumps, five kernels, batch 16
W_DISCONTINUOUS = 3     # disk / square indicators (Fourier smoothing)
W_LIPPMANN = 4          # contrasts for the Lippmann-Schwinger solve
W_SERVING = 5           # request mix


def seed_for(workload: int, n: int, item: int = 0) -> int:
    return 10**6 * workload + 10**3 * int(round(math.log2(max(n, 1)))) + item


def grid(n):
    x = np.arange(n, dtype=np.float64) / n
    return np.meshgrid(x, x, indexing="ij")


def _add_bump(out, n, c1, c2, R, amp):
    """out += amp * exp(-1 / (1 - r^2/R^2)) for r = |x - c| < R, evaluated on its bounding box."""
    lo1, hi1 = max(0, int(math.floor((c1 - R) * n))), min(n, int(math.ceil((c1 + R) * n)) + 1)
    lo2, hi2 = max(0, int(math.floor((c2 - R) * n))), min(n, int(math.ceil((c2 + R) * n)) + 1)
    if lo1 >= hi1 or lo2 >= hi2:
        return
    x1 = np.arange(lo1, hi1, dtype=np.float64)[:, None] / n - c1
    x2 = np.arange(lo2, hi2, dtype=np.float64)[None, :] / n - c2
    t = (x1 * x1 + x2 * x2) / (R * R)
    inside = t < 1.0
    v = np.zeros_like(t)
    v[inside] = np.exp(-1.0 / (1.0 - t[inside]))
    out[lo1:hi1, lo2:hi2] += amp * v


def bump(n, centre=(0.5, 0.5), R=0.4, amp=1.0):
    """exp(-1/(1 - |x-c|^2/R^2)) inside the disk of radius R (peak e^-1), 0 outside."""
    out = np.zeros((n, n))
    _add_bump(out, n, centre[0], centre[1], R, amp)
    return out


def poisson_bump(n=64):
    """Single bump of radius 0.4 at (0.5, 0.5)."""
    return bump(n, (0.5, 0.5), 0.4)


def bump_sum_params(rng):
    K = int(rng.integers(1, 9))
    c = rng.uniform(0.2, 0.8, size=(K, 2))
    r = rng.uniform(0.05, 0.2, size=K)
    amp = rng.standard_normal(K)
    return c, r, amp


def bump_sums(n, batch, seed=None, dtype=np.float64):
    """batch densities, each a sum of K ~ U{1..8} bumps: centres U[0.2,0.8]^2,
    radii U[0.05,0.2], amplitudes N(0,1)."""
    rng = np.random.default_rng(seed_for(W_KERNEL_SWEEP, n) if seed is None else seed)
    out = np.zeros((batch, n, n), dtype=np.float64)
    for i in range(batch):
        c, r, amp = bump_sum_params(rng)
        for k in range(len(r)):
            _add_bump(out[i], n, c[k, 0], c[k, 1], r[k], amp[k])
    return out.astype(dtype, copy=False)


def gaussian(n, centre=(0.5, 0.5), sigma=0.05):
    """(1/(2 pi sigma^2)) exp(-|x-c|^2 / (2 sigma^2))."""
    X1, X2 = grid(n)
    r2 = (X1 - centre[0]) ** 2 + (X2 - centre[1]) ** 2
    return np.exp(-r2 / (2 * sigma * sigma)) / (2 * math.pi * sigma * sigma)


def polynomial_density(n, m):
    """(x1(1-x1) x2(1-x2))^m."""
    X1, X2 = grid(n)
    return (X1 * (1 - X1) * X2 * (1 - X2)) ** m


def polynomial_laplacian(n, m):
    """Laplacian of (x1(1-x1) x2(1-x2))^m."""
    X1, X2 = grid(n)
    P1, P2 = X1 * (1 - X1), X2 * (1 - X2)

    def d2(P, t):
        return m * (m - 1) * P ** (m - 2) * (1 - 2 * t) ** 2 - 2 * m * P ** (m - 1)
    return d2(P1, X1) * P2 ** m + P1 ** m * d2(P2, X2)


def gaussian_sum(n, alpha, centres):
    X1, X2 = grid(n)
    return sum(np.exp(-alpha * ((X1 - c1) ** 2 + (X2 - c2) ** 2)) for c1, c2 in centres)


def gaussian_sum_laplacian(n, alpha, centres):
    """Laplacian of gaussian_sum: sum (4 alpha^2 |x-c|^2 - 4 alpha) exp(-alpha |x-c|^2)."""
    X1, X2 = grid(n)
    out = np.zeros((n, n))
    for c1, c2 in centres:
        r2 = (X1 - c1) ** 2 + (X2 - c2) ** 2
        out += (4 * alpha * alpha * r2 - 4 * alpha) * np.exp(-alpha * r2)
    return out


def yukawa_source(n, kappa, delta=0.08, centre=(0.5, 0.5)):
    """f = ((-4 r^2 + 4 delta^2)/delta^4 + kappa^2) exp(-r^2/delta^2), r = |x - centre|: the right-hand
    side whose solution of -Delta u + kappa^2 u = f is yukawa_solution."""
    X1, X2 = grid(n)
    r2 = (X1 - centre[0]) ** 2 + (X2 - centre[1]) ** 2
    return ((-4.0 * r2 + 4.0 * delta * delta) / delta ** 4 + kappa * kappa) * np.exp(-r2 / (delta * delta))


def yukawa_solution(n, delta=0.08, centre=(0.5, 0.5)):
    """exp(-|x - centre|^2 / delta^2)."""
    X1, X2 = grid(n)
    return np.exp(-((X1 - centre[0]) ** 2 + (X2 - centre[1]) ** 2) / (delta * delta))


def indicator_rect(n, x0, x1, y0, y1):
    """Grid samples of the indicator of [x0,x1] x [y0,y1]: 1 inside, 1/2 on an edge node,
    1/4 on a corner node (trapezoidal convention at ties)."""
    x = np.arange(n, dtype=np.float64) / n

    def axis(lo, hi):
        v = ((x > lo) & (x < hi)).astype(np.float64)
        v[np.isclose(x, lo, rtol=0, atol=1e-14) | np.isclose(x, hi, rtol=0, atol=1e-14)] = 0.5
        return v

    return np.outer(axis(x0, x1), axis(y0, y1))


def indicator_disk(n, centre=(0.5, 0.5), r=0.3):
    X1, X2 = grid(n)
    d = np.hypot(X1 - centre[0], X2 - centre[1])
    out = (d < r).astype(np.float64)
    out[np.isclose(d, r, rtol=0, atol=1e-14)] = 0.5
    return out


def smooth_extension(n, seed=None):
    """Smooth positive factor u~ for the disk workload: a bump of radius 0.5 centred at a
    seeded point of [0.4, 0.6]^2 (positive on the disk of radius 0.3 about (0.5, 0.5))."""
    rng = np.random.default_rng(seed_for(W_DISCONTINUOUS, n) if seed is None else seed)
    c = rng.uniform(0.4, 0.6, size=2)
    return bump(n, (c[0], c[1]), 0.5)


def lippmann_contrast(n, kind="bump"):
    """Contrast m = 0.5 * bump(radius 0.4) or 0.5 * disk indicator (radius 0.3), centred."""
    if kind == "bump":
        return 0.5 * bump(n, (0.5, 0.5), 0.4)
    if kind == "disk":
        return 0.5 * indicator_disk(n, (0.5, 0.5), 0.3)
    raise ValueError(kind)


def _radius(n, centre=(0.5, 0.5)):
    X1, X2 = grid(n)
    return np.hypot(X1 - centre[0], X2 - centre[1])


def _half_window(t):
    """exp(2 e^{-1/t} / (t - 1)) on (0, 1), 1 at t <= 0, 0 at t >= 1 (the half-window that the
    smooth disc's refractive index is built with)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t <= 0.0, 1.0, 0.0)
    mid = (t > 0.0) & (t < 1.0)
    tm = t[mid]
    out[mid] = np.exp(2.0 * np.exp(-1.0 / tm) / (tm - 1.0))
    return out


def smooth_disc_contrast(n, t1=0.45, centre=(0.5, 0.5)):
    """m = 1 - mu for the disc with smooth refractive index: mu = 2 for r <= t0 = 0.9 t1,
    1 + varkappa((r - t0)/(t1 - t0)) for t0 < r < t1, 1 beyond (its diameter 2 t1 = 0.9)."""
    r = _radius(n, centre)
    t0 = 0.9 * t1
    mu = np.where(r <= t0, 2.0, np.where(r < t1, 1.0 + _half_window((r - t0) / (t1 - t0)), 1.0))
    return 1.0 - mu


def filter_disc_contrast(n, a=0.5, centre=(0.5, 0.5)):
    """m = -exp(-(1/2) (2 r / a)^8): the smooth filter disc of diameter a."""
    r = _radius(n, centre)
    return -np.exp(-0.5 * (2.0 * r / a) ** 8)


def luneburg_contrast(n, a=0.9, centre=(0.5, 0.5)):
    """m = (2 r / a)^2 - 1 inside the Luneburg lens of diameter a, 0 outside."""
    r = _radius(n, centre)
    return np.where(r < 0.5 * a, (2.0 * r / a) ** 2 - 1.0, 0.0)


def plane_wave(n, kappa, angle=0.0):
    """u_inc(x) = exp(i kappa (x1 cos angle + x2 sin angle)) on the grid (angle 0: exp(i kappa x1))."""
    X1, X2 = grid(n)
    if angle == 0.0:
        return np.exp(1j * kappa * X1)
    return np.exp(1j * kappa * (X1 * np.cos(angle) + X2 * np.sin(angle)))


SERVING_SIZES = (128, 256, 512, 1024, 2048)
SERVING_WEIGHTS = (0.3, 0.3, 0.2, 0.15, 0.05)
SWEEP_KERNELS = (("log", {}), ("pow", {"gamma": -0.5}), ("pow", {"gamma": -1.0}),
                 ("pow", {"gamma": -1.5}), ("helmholtz", {"kappa": 20.0}))


def serving_requests(count, rate=200.0, seed=None, ls_fraction=0.5, sizes=SERVING_SIZES,
                     weights=SERVING_WEIGHTS):
    """Poisson arrivals (mean `rate`/s) of convolution and Lippmann-Schwinger requests:
    n drawn from `sizes` with `weights`, kernel from the five-kernel sweep, kappa ~ U[5, 60]."""
    rng = np.random.default_rng(10**6 * W_SERVING if seed is None else seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = []
    for i in range(count):
        n = int(rng.choice(sizes, p=weights))
        is_ls = bool(rng.uniform() < ls_fraction)
        kappa = float(rng.uniform(5.0, 60.0))
        kern = SWEEP_KERNELS[int(rng.integers(0, len(SWEEP_KERNELS)))]
        reqs.append({"id": i, "t_arrival": float(t[i]), "n": n, "kind": "ls" if is_ls else "conv",
                     "kernel": kern[0], "params": dict(kern[1]), "kappa": kappa,
                     "seed": seed_for(W_SERVING, n, i)})
    return reqs
