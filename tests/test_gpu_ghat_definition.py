"""The GPU's moment table against quadrature of the moments' definition, eq. (ghat) of Sec. 2.2,
at the n = 4096, b = 3 table's own entries (M b = 12288, |k| up to 6144 sqrt 2, z = s a up to
3.1e4), without passing through any oracle code: the reference values in
tests/golden/ghat_quadrature.txt are 20-digit mpmath quadratures of 2 pi int_0^a g J0 rho d rho
(written by tests/golden/make_ghat_quadrature.py).  The entries straddle every switch of the
GPU's moment kernel and of the oracle's: z = 45 and 60 for |x|^gamma, the 5 % and 8 % bands
around s = kappa for the Helmholtz kernel.

Tolerance: 1e-13 of the table's largest entry (1e-12 for the Helmholtz kernel, as in
test_ghat_table_matches_oracle: within ~10 % of s = kappa the closed form's numerator cancels
about two digits, which the device J0, J1 and their absolute error ~1e-16 at z ~ 35 make
~1e-12 of the entry; inside the 8 % band the quadrature sums ~2000 device J0 values), and
1e-10 relative for entries above 1e-6 of it.
"""
import math

import numpy as np
import pytest
from conftest import load_golden

from paper_2107_03958_gb300.api import ConvPlan

pytestmark = pytest.mark.gpu

FAMILY = {0: "log", 1: "pow", 2: "helmholtz"}


def _rows():
    rows = load_golden("ghat_quadrature.txt")
    groups = {}
    for fam, gamma, kappa, k1, k2, re, im in rows:
        groups.setdefault((int(fam), gamma, kappa), []).append((int(k1), int(k2), complex(re, im)))
    return groups


GROUPS = _rows()


@pytest.mark.parametrize("key", sorted(GROUPS), ids=lambda k: "%s-%g-%g" % (FAMILY[k[0]], k[1], k[2]))
def test_ghat_table_matches_quadrature_of_the_definition(key):
    fam, gamma, kappa = key
    kernel = FAMILY[fam]
    plan = ConvPlan(kernel, n=4096, period=3, precision="fp64", io="r2r" if kernel != "helmholtz" else "r2c",
                    gamma=gamma, kappa=kappa, scale=1.0)
    table = plan.ghat_quadrant()
    g0 = np.max(np.abs(table))
    for k1, k2, ref in GROUPS[key]:
        for got in (table[k2, k1], table[k1, k2]):
            err = abs(got - ref)
            assert err <= (1e-12 if kernel == "helmholtz" else 1e-13) * g0, (k1, k2, got, ref, err / g0)
            if abs(ref) > 1e-6 * g0:
                assert err <= 1e-10 * abs(ref), (k1, k2, got, ref, err / abs(ref))
