"""Power-spectrum wedges from the multipoles (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 5 of the paper replaces the Legendre weight of the estimator by top hats in mu,
0 <= mu <= 1/2 (P_perp) and 1/2 < mu <= 1 (P_para), and approximates both by the
first three even multipoles (Eqs. 16-17): the coefficients are the averages of L_2
and L_4 over each half of the mu range.

Pinned by: the coefficients against numerical averages of the Legendre polynomials
over the two ranges, and the exact wedges of a P(k, mu) that is a polynomial of
degree 4 in mu (for which the truncation at l = 4 is exact).
"""
from __future__ import annotations

import numpy as np


def wedges_from_multipoles(p0, p2, p4):
    """(P_perp, P_para) of Eqs. 16-17."""
    p0, p2, p4 = (np.asarray(a, dtype=np.float64) for a in (p0, p2, p4))
    return p0 - 3.0 / 8.0 * p2 + 15.0 / 128.0 * p4, p0 + 3.0 / 8.0 * p2 - 15.0 / 128.0 * p4
