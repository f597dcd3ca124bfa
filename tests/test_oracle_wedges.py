"""Pins of the wedges: the combination of Eqs. 16-17 and the direct-sum definition of
Eqs. 14-15."""
import math

import numpy as np
from numpy.polynomial import legendre

import oracle
import synth
from oracle.binning import BinSpec
from oracle.wedges import wedges_from_multipoles, wedges_sum_gal


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


# --------------------------------------------------------------------------
# Eqs. 14-15 by their definition (direct sum)
# --------------------------------------------------------------------------



def test_direct_wedges_partition_the_monopole():
    """The two top hats add up to one: P_perp + P_para = 2 P_0 of the galaxy sum."""
    gal, ran, geo = synth.poisson_cube(400, 2000, side=300.0, center=(100.0, -250.0, 400.0), seed=31)
    bins = BinSpec.up_to(np.pi * 16 / geo.box_len, 0.01)
    wd = wedges_sum_gal(gal, ran, geo, 16, bins)
    ref = oracle.sum_gal(gal, ran, geo, 16, bins, ell_max=0)
    has = ref.n_modes > 0
    raw = ref.sum0[has] / ref.n_modes[has] / ref.norm.I
    np.testing.assert_array_equal(wd.n_modes, ref.n_modes)
    assert np.max(np.abs(wd.p_perp[has] + wd.p_para[has] - 2 * ref.p0[has]) / raw) < 1e-12
    # and both wedges differ from P_0 (the LOS varies across this catalogue)
    assert np.max(np.abs(wd.p_perp[has] - ref.p0[has]) / raw) > 1e-3


def _lattice_counts(n, box_len, bins, rvec):
    """Hermitian-weighted mode counts per shell with |k_hat . r_hat| <= 1/2, and all
    modes, by enumerating integer vectors of the n^3 half grid (integers only, except
    |k| for the shell index)."""
    kf = 2 * math.pi / box_len
    knyq = kf * n / 2
    perp = np.zeros(bins.n_bins)
    total = np.zeros(bins.n_bins)
    half = [m for m in range(-n // 2, n // 2)]
    r2 = float(np.dot(rvec, rvec))
    for mx in half:
        for my in half:
            for mz in range(0, n // 2 + 1):
                m2 = mx * mx + my * my + mz * mz
                kk = kf * math.sqrt(m2)
                if m2 == 0 or kk >= knyq:
                    continue
                b = math.floor((kk - bins.k_min) / bins.dk)
                if not 0 <= b < bins.n_bins:
                    continue
                hw = 2.0 if 0 < mz < n // 2 else 1.0
                dot = mx * rvec[0] + my * rvec[1] + mz * rvec[2]
                total[b] += hw
                if 4.0 * dot * dot <= m2 * r2:
                    perp[b] += hw
    return perp, total


def test_direct_wedges_one_particle_is_a_direction_count():
    """One particle of unit net weight (a galaxy of weight 7/4 and a random of weight 1
    at the same point, alpha = 3/4): A_0 = e^{-i phi} and B_perp = Theta A_0, so each
    mode adds its top hat, and the shell sums count the lattice directions within 60
    degrees of perpendicular to the particle's line of sight."""
    pos = np.array([[330.0, -71.5, -20.0]], dtype=np.float32)  # LOS mostly along x: mu < -1/2 occurs
    gal = synth.Catalog.from_positions(pos, 1.75, 1e-4)
    ran = synth.Catalog.from_positions(pos, 1.0, 1e-4)
    geo = synth.Geometry((-200.0, -200.0, -200.0), 600.0, (10.0, 20.0, -30.0))
    bins = BinSpec.up_to(np.pi * 12 / geo.box_len, 0.004)
    wd = wedges_sum_gal(gal, ran, geo, 12, bins, alpha=0.75)
    rvec = pos[0].astype(np.float64) - np.asarray(geo.observer)
    perp, total = _lattice_counts(12, geo.box_len, bins, rvec)
    np.testing.assert_array_equal(wd.n_modes, total)
    np.testing.assert_allclose(wd.sum_perp, perp, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(wd.sum_para, total - perp, rtol=1e-12, atol=1e-12)
    has = total > 0
    I, S = wd.norm.I, wd.norm.S
    np.testing.assert_allclose(wd.p_perp[has], 2.0 / I * perp[has] / total[has] - S / I, rtol=1e-12)


def test_direct_wedges_distant_observer_use_the_mode_direction():
    """An observer 1e8 Mpc/h away along -z: every particle's mu is k_hat_z (to 1e-6), so
    B_perp = Theta(|k_hat_z| <= 1/2) A_0 mode by mode (no integer vector has
    |k_hat_z| = 1/2 exactly: x^2 + y^2 = 3 z^2 has no solution but 0)."""
    gal, ran, geo = synth.poisson_cube(300, 1500, side=400.0, center=(0.0, 0.0, 0.0), seed=32)
    geo = synth.Geometry(geo.box_min, geo.box_len, (0.0, 0.0, -1.0e8))
    n = 16
    bins = BinSpec.up_to(np.pi * n / geo.box_len, 0.01)
    wd = wedges_sum_gal(gal, ran, geo, n, bins)
    ref = oracle.sum_gal(gal, ran, geo, n, bins, ell_max=0)
    from oracle.direct import _valid_modes
    M, bidx, w, _, _ = _valid_modes(n, geo.box_len, bins)
    A0 = ref.modes[0]
    kz = np.abs(M[:, 2]) / np.linalg.norm(M, axis=1)
    assert np.min(np.abs(kz - 0.5)) > 1e-4
    want = np.bincount(bidx, weights=w * np.abs(A0) ** 2 * (kz <= 0.5), minlength=bins.n_bins)
    scale = np.max(ref.sum0)
    assert np.max(np.abs(wd.sum_perp - want)) < 1e-10 * scale
