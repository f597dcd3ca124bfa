"""Pins of the wedge combination (Eqs. 16-17)."""
import numpy as np
from numpy.polynomial import legendre

from oracle.wedges import wedges_from_multipoles


def _mean_over(f, a, b, n=200_001):
    x = np.linspace(a, b, n)
    y = f(x)
    return np.trapezoid(y, x) / (b - a) if hasattr(np, "trapezoid") else np.trapz(y, x) / (b - a)


def test_coefficients_are_legendre_averages_over_each_half():
    L2 = lambda mu: legendre.legval(mu, [0, 0, 1])
    L4 = lambda mu: legendre.legval(mu, [0, 0, 0, 0, 1])
    perp, para = wedges_from_multipoles(1.0, 0.0, 0.0)
    assert perp == 1.0 and para == 1.0
    perp, para = wedges_from_multipoles(0.0, 1.0, 0.0)
    assert abs(perp - _mean_over(L2, 0.0, 0.5)) < 1e-10 and abs(para - _mean_over(L2, 0.5, 1.0)) < 1e-10
    perp, para = wedges_from_multipoles(0.0, 0.0, 1.0)
    assert abs(perp - _mean_over(L4, 0.0, 0.5)) < 1e-10 and abs(para - _mean_over(L4, 0.5, 1.0)) < 1e-10


def test_exact_for_a_degree_four_spectrum():
    # Kaiser-like P(mu) = b^2 (1 + beta mu^2)^2 P_lin: multipoles up to l = 4 only
    b, beta, plin = 1.9, 0.37, 12_000.0
    P = lambda mu: b * b * (1 + beta * mu * mu) ** 2 * plin
    mu = np.linspace(-1, 1, 40_001)
    c = legendre.legfit(mu, P(mu), 6)
    p0, p2, p4 = c[0], c[2], c[4]
    assert abs(c[6]) < 1e-6 * p0
    perp, para = wedges_from_multipoles(p0, p2, p4)
    assert abs(perp - _mean_over(P, 0.0, 0.5)) < 1e-8 * p0
    assert abs(para - _mean_over(P, 0.5, 1.0)) < 1e-8 * p0
