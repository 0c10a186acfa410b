"""Writes ghat_quadrature.txt: moments ghat(k) of eq. (ghat), Sec. 2.2, by 20-digit quadrature of
their definition (oracle/quad_mp.py), at table entries (k1, k2) of the n = 4096, b = 3 plan
(M b = 12288, default truncation radius a = (sqrt 2 + 2)/2), unscaled kernels:
  |x|^gamma, gamma in {-1/2, -1, -3/2}: both sides of z = s a = 45 and 60, and up to the table's
      largest |k| (z ~ 3.1e4);
  (i/4) H0^(1)(20 |x|): both sides of the resonance bands |s - kappa| < 5% and 8% of kappa, and
      large |k|;
  log|x|: k = 0, a moderate and the largest |k|.
Run once (about 10 minutes on 8 cores): python tests/golden/make_ghat_quadrature.py
"""
import math
import multiprocessing as mpc
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

B = 3.0
A = 0.5 * (math.sqrt(2.0) + B - 1.0)
POW_K = [(12, 3), (13, 1), (16, 4), (17, 3), (100, 37), (1000, 0), (4000, 3000), (6144, 6144)]
HELM_K = [(9, 0), (8, 4), (9, 3), (7, 7), (10, 1), (10, 3), (300, 200), (6144, 6144)]
LOG_K = [(0, 0), (37, 11), (6144, 6144)]


def jobs():
    out = []
    for g in (-0.5, -1.0, -1.5):
        out += [("pow", g, 0.0, k) for k in POW_K]
    out += [("helm", 0.0, 20.0, k) for k in HELM_K]
    out += [("log", 0.0, 0.0, k) for k in LOG_K]
    return out


def run(job):
    from oracle import quad_mp
    kind, gamma, kappa, (k1, k2) = job
    v = quad_mp.ghat_quadrature(kind, math.hypot(k1, k2), B, A, gamma=gamma, kappa=kappa)
    return kind, gamma, kappa, k1, k2, v


if __name__ == "__main__":
    with mpc.get_context("spawn").Pool(os.cpu_count()) as pool:
        rows = pool.map(run, jobs(), chunksize=1)
    with open(os.path.join(HERE, "ghat_quadrature.txt"), "w") as f:
        f.write("# ghat(k) = 2 pi int_0^a g(rho) J0(2 pi |k| rho / b) rho d rho (eq. (ghat), Sec. 2.2) by\n")
        f.write("# 20-digit quadrature of the definition (oracle/quad_mp.py, written by make_ghat_quadrature.py)\n")
        f.write("# b = 3, a = (sqrt 2 + 2)/2; unscaled g: 0 = log|x|, 1 = |x|^gamma, 2 = (i/4) H0^(1)(kappa |x|)\n")
        f.write("# family gamma kappa k1 k2 re im\n")
        fam = {"log": 0, "pow": 1, "helm": 2}
        for kind, gamma, kappa, k1, k2, v in rows:
            f.write("%d %.2f %.1f %d %d %.17e %.17e\n" % (fam[kind], gamma, kappa, k1, k2, v.real, v.imag))
