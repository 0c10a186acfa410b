"""Pins of the oracle's moments without a closed form (Sec. 2.3) and of the Yukawa kernel
(Sec. 3.2) to values fixed by the paper and by mathematics (no GPU).

  - K0, K1 against mpmath; the Yukawa moments' closed form against 20-digit quadrature of their
    definition (oracle/quad_mp.py);
  - the Clenshaw-Curtis rule of eq. (cc_pts)/(cc_wts) integrates polynomials exactly;
  - moments by the quadrature of Sec. 2.3 equal the closed forms of Sec. 2.2;
  - the Yukawa solve reproduces Table 9 (closed-form and quadrature moments);
  - the localized scheme, eq. (io_split), reproduces Tables 4 and 5 on the finer grids.
"""
import math

import numpy as np
import pytest
from conftest import load_golden

import oracle as O
from paper_2107_03958_gb300 import inputs

A3 = O.default_trunc_radius(3.0)


def test_bessel_k_matches_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x in (1e-8, 1e-3, 0.2, 1.0, 1.9, 2.0, 2.1, 5.0, 34.1, 120.0, 341.4, 700.0):
        for nu in (0, 1):
            ref = float(mp.besselk(nu, x))
            assert abs(O.bessel_k(nu, x) - ref) <= 2e-14 * ref, (nu, x)


def test_yukawa_moment_matches_quadrature_of_definition():
    pytest.importorskip("mpmath")
    from oracle import quad_mp
    for kappa in (1.0, 20.0, 200.0):
        for k in (0.0, 1.0, 7.3, 40.0):
            ref = quad_mp.ghat_quadrature("yukawa", k, 3.0, A3, kappa=kappa).real
            got = O.ghat_radial("yukawa", k, 3.0, A3, kappa=kappa)
            scale = abs(O.ghat_radial("yukawa", 0.0, 3.0, A3, kappa=kappa))
            assert abs(got - ref) <= 1e-13 * scale, (kappa, k, got, ref)


@pytest.mark.parametrize("npc", [8, 17, 64])
def test_cc_rule_integrates_polynomials(npc):
    """The rule of eq. (cc_pts)/(cc_wts) on [0, alpha] is interpolatory on npc points: exact for
    every polynomial of degree < npc (and odd-symmetric ones beyond)."""
    alpha = 1.37
    x, w = O.cc_rule(npc, alpha)
    assert np.all((x > 0) & (x < alpha))
    for deg in range(npc):
        exact = alpha ** (deg + 1) / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) <= 1e-13 * max(1.0, exact), deg


@pytest.mark.parametrize("kind,kw", [("log", {"scale": -1 / (2 * math.pi)}), ("pow", {"gamma": -0.5}),
                                     ("pow", {"gamma": -1.5}), ("helm", {"kappa": 20.0}),
                                     ("yukawa", {"kappa": 1.0}), ("yukawa", {"kappa": 200.0})])
def test_numeric_moments_match_closed_forms(kind, kw):
    """Sec. 2.3's quadrature after rho = tau^4 with 1024 points of eq. (cc_pts)/(cc_wts) gives the
    Sec. 2.2 moments of every table entry at M = 96."""
    M = 96
    cf = O.ghat_full(kind, M, 3.0, A3, **kw)
    nm = O.ghat_numeric_full(kind, M, 3.0, A3, p=4, npc=1024, **kw)
    assert np.max(np.abs(nm - cf)) <= 2e-14 * np.max(np.abs(cf))


def test_eta_window():
    beta = 0.8
    assert O.eta(0.0, beta) == 1.0 and O.eta(0.4, beta) == 1.0 and O.eta(0.8, beta) == 0.0
    r = np.linspace(0.4, 0.8, 401)
    e = np.array([O.eta(x, beta) for x in r])
    assert np.all(np.diff(e) <= 0) and np.all((e >= 0) & (e <= 1))
    # flat to all orders at both ends of the transition
    assert 1.0 - O.eta(0.41, beta) < 1e-16 and O.eta(0.799, beta) < 1e-60


@pytest.mark.parametrize("col,kappa", [(1, 1.0), (2, 200.0)])
def test_table9_yukawa(col, kappa):
    """Table 9: g = K0(kappa|x|)/(2 pi) applied to f gives u; eps_n within a factor 2 of the printed
    column for n = 4..32 and at round-off (< 2e-15) at n = 64, with closed-form moments and with
    the quadrature moments of Sec. 2.3."""
    tab = load_golden("table9_yukawa.txt")
    for row in tab:
        n = int(row[0])
        M = 3 * n
        f = inputs.yukawa_source(n, kappa)
        u = inputs.yukawa_solution(n)
        for g in (O.ghat_full("yukawa", M, 3.0, A3, kappa=kappa),
                  O.ghat_numeric_full("yukawa", M, 3.0, A3, kappa=kappa, npc=2048)):
            e = O.rel_err(u, O.conv(f, M, g).real)
            if n <= 32:
                assert 0.5 < e / row[col] < 2.0, (n, e, row[col])
            else:
                assert e < 2e-15, (n, e)


def _fine_reference(kind, kw, dens, nf):
    Mf = 3 * nf
    return O.conv(dens(nf), Mf, O.ghat_full(kind, Mf, 3.0, A3, **kw)).real


def _localized_errors(kind, kw, dens, ns, nf, beta=1.0):
    ref = _fine_reference(kind, kw, dens, nf)
    out = []
    for n in ns:
        g = O.ghat_localized_full(kind, n, 3.0, A3, beta, p=4, npc=4096, **kw)
        c = O.conv(dens(n), 3 * n, g).real
        out.append(O.rel_err(ref[::nf // n, ::nf // n], c))
    return np.array(out)


KERNELS = [("pow", {"gamma": -0.5}), ("pow", {"gamma": -1.0}), ("pow", {"gamma": -1.5}), ("log", {})]


@pytest.mark.parametrize("col", range(4))
def test_table4_localized_kernels(col):
    """Table 4: the localized scheme (beta = 1), u = (x1(1-x1)x2(1-x2))^3; eps_n within a factor 2
    of the printed values for n = 64, 128 (the coarse-grid values depend on the unprinted beta)."""
    tab = load_golden("table4_localized_kernels.txt")
    rows = tab[(tab[:, 0] >= 64) & (tab[:, 0] <= 128)]
    kind, kw = KERNELS[col]
    errs = _localized_errors(kind, kw, lambda n: inputs.polynomial_density(n, 3), rows[:, 0].astype(int), 512)
    ratio = errs / rows[:, 1 + col]
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_table5_localized_smoothness(m):
    """Table 5: the localized scheme, |x|^-1, u = (x1(1-x1)x2(1-x2))^m; eps_n within a factor 2 of
    the printed values for n = 64, 128."""
    tab = load_golden("table5_localized_smoothness.txt")
    rows = tab[(tab[:, 0] >= 64) & (tab[:, 0] <= 128)]
    errs = _localized_errors("pow", {"gamma": -1.0}, lambda n: inputs.polynomial_density(n, m),
                             rows[:, 0].astype(int), 512)
    ratio = errs / rows[:, m]
    assert np.all((ratio > 0.5) & (ratio < 2.0)), ratio


def test_localized_multiplier_converges_to_the_global_scheme():
    """On a fine grid the localized and the global scheme give the same A_n u up to the
    discretisation error of either (Sec. 2.3: localization loses no accuracy)."""
    n = 128
    u = inputs.polynomial_density(n, 3)
    glob = O.conv(u, 3 * n, O.ghat_full("log", 3 * n, 3.0, A3)).real
    loc = O.conv(u, 3 * n, O.ghat_localized_full("log", n, 3.0, A3, 1.0, npc=4096)).real
    assert O.rel_err(glob, loc) < 2e-8
