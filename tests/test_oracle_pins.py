"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests needs a GPU.  Each one is chosen so that a plausible slip in
the oracle (a dropped or mis-indexed term of Eq. 12, a wrong sign of the interlacing
phase, a wrong window power, a wrong normalisation) makes it fail.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.integrate

import oracle
import synth
from oracle.assignment import _stencil
from oracle.binning import BinSpec, half_modes, mode_bins
from oracle.estimator import node_offsets, window
from oracle.terms import A2_TERMS, A4_TERMS, A6_TERMS, field_monomial

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    m = np.isfinite(a) & np.isfinite(b)
    scale = np.max(np.abs(a[m])) if np.any(m) else 1.0
    return float(np.max(np.abs(a[m] - b[m])) / scale)


# --------------------------------------------------------------------------
# Eqs. (10) and (12) as data
# --------------------------------------------------------------------------

def test_terms_match_printed_equations():
    """The oracle's term tables equal the printed Eqs. (10) and (12)."""
    rows = []
    with open(os.path.join(GOLDEN, "eq10_eq12_terms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            eq, c, px, py, pz, name = line.split()
            rows.append((eq, int(c), (int(px), int(py), int(pz)), name))
    assert [(c, p, n) for e, c, p, n in rows if e == "A2"] == A2_TERMS
    assert [(c, p, n) for e, c, p, n in rows if e == "A4"] == A4_TERMS


@pytest.mark.parametrize("terms,deg", [(A2_TERMS, 2), (A4_TERMS, 4), (A6_TERMS, 6)])
def test_terms_expand_mu_power(terms, deg):
    """sum_terms coef k^p r^m / (k^n r^n) == (k_hat . r_hat)^n on random vectors
    (the decomposition is exact, Sec. 3)."""
    rng = np.random.default_rng(11)
    k = rng.standard_normal((200, 3))
    r = rng.standard_normal((200, 3))
    mu = np.sum(k * r, axis=1) / np.linalg.norm(k, axis=1) / np.linalg.norm(r, axis=1)
    acc = np.zeros(200)
    for coef, kp, name in terms:
        (a, b, c), d = field_monomial(name)
        assert d == deg
        acc += coef * np.prod(k ** np.array(kp), axis=1) * r[:, 0] ** a * r[:, 1] ** b * r[:, 2] ** c
    acc /= np.linalg.norm(k, axis=1) ** deg * np.linalg.norm(r, axis=1) ** deg
    np.testing.assert_allclose(acc, mu ** deg, rtol=1e-12, atol=1e-12)
    # every term's k monomial equals its field's r monomial (same multi-index)
    for coef, kp, name in terms:
        assert tuple(kp) == field_monomial(name)[0]
        assert coef == math.factorial(deg) // np.prod([math.factorial(v) for v in kp])


# --------------------------------------------------------------------------
# Normalisation and binning
# --------------------------------------------------------------------------

def test_norm_closed_form():
    gal, ran, geo = synth.poisson_cube(2000, 10000, seed=1)
    nm = oracle.catalog_sums(gal, ran)
    ref = {}
    with open(os.path.join(GOLDEN, "cube32_normalisation.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            ref[k] = float(v)
    assert nm.alpha == pytest.approx(ref["alpha"], rel=1e-15)
    assert nm.I == pytest.approx(ref["I"], rel=1e-6)   # nbar stored in float32
    assert nm.S == pytest.approx(ref["S"], rel=1e-15)
    assert nm.S / nm.I == pytest.approx(ref["S_over_I"], rel=1e-6)


@pytest.mark.parametrize("n", [8, 12, 16])
def test_half_mode_weights(n):
    """Hermitian weights on the half grid reproduce the full-grid count per bin."""
    L = 100.0
    bins = BinSpec(0.0, 0.05, 12)
    bidx, w, _ = mode_bins(n, L, bins)
    half = np.bincount(bidx[bidx >= 0], weights=w[bidx >= 0], minlength=bins.n_bins)
    m = np.fft.fftfreq(n, d=1.0 / n)
    full = np.zeros(bins.n_bins)
    kf = 2 * np.pi / L
    for a, b, c in itertools.product(m, m, m):
        m2 = a * a + b * b + c * c
        kk = kf * math.sqrt(m2)
        if m2 == 0 or kk >= kf * n / 2:
            continue
        bb = math.floor((kk - bins.k_min) / bins.dk)
        if 0 <= bb < bins.n_bins:
            full[bb] += 1
    np.testing.assert_array_equal(half, full)


# --------------------------------------------------------------------------
# Assignment and window
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["ngp", "cic", "tsc"])
@pytest.mark.parametrize("interlaced", [False, True])
def test_mass_conservation(kind, interlaced):
    gal, ran, geo = synth.poisson_cube(500, 2500, seed=5)
    nm = oracle.catalog_sums(gal, ran)
    F = oracle.assign_mesh(gal, ran, nm.alpha, geo.box_min, geo.box_len, 16, kind, interlaced)
    assert np.sum(F) == pytest.approx(nm.sum_w_gal - nm.alpha * nm.sum_w_ran, abs=1e-9)


@pytest.mark.parametrize("kind", ["ngp", "cic", "tsc"])
@pytest.mark.parametrize("interlaced", [False, True])
def test_c_deposit_matches_numpy(kind, interlaced):
    """The plain-C deposit loop equals the numpy deposit (same definitions)."""
    import oracle.cbuild
    oracle.cbuild.build()
    gal, ran, geo = synth.poisson_cube(700, 3500, seed=8)
    a = oracle.assign_mesh(gal, ran, 0.2, geo.box_min, geo.box_len, 16, kind, interlaced, impl="numpy")
    b = oracle.assign_mesh(gal, ran, 0.2, geo.box_min, geo.box_len, 16, kind, interlaced, impl="c")
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["ngp", "cic", "tsc"])
def test_window_is_kernel_transform(kind):
    """window() equals the Fourier transform of the assignment kernel that
    ``_stencil`` defines, integrated numerically (continuum, unit cell)."""
    def kernel(d):
        # weight the stencil gives to a node at offset d from the particle
        best = 0.0
        for off, wt in _stencil(np.array([-d + 0.0]), kind):
            if abs(off[0] - 0.0) < 1e-12:
                best += wt[0]
        return best

    n = 16
    Wk = window(n, kind)
    for m in range(1, n // 2):
        k = 2 * np.pi * m / n
        val, _ = scipy.integrate.quad(lambda d: kernel(d) * math.cos(k * d), -1.5, 1.5,
                                      points=[-1.0, -0.5, 0.0, 0.5, 1.0], limit=200)
        assert Wk[m, 0, 0] == pytest.approx(val, rel=1e-9)
        assert Wk[0, m, 0] == pytest.approx(val, rel=1e-9)
        assert Wk[0, 0, m] == pytest.approx(val, rel=1e-9)


@pytest.mark.parametrize("kind,closed", [
    ("ngp", lambda s: np.ones_like(s)),
    ("cic", lambda s: 1 - 2.0 / 3.0 * s ** 2),
    ("tsc", lambda s: 1 - s ** 2 + 2.0 / 15.0 * s ** 4),
])
def test_poisson_shot_noise_shape(kind, closed):
    """Unclustered points in the periodic box: E|A_0(k)|^2 = S prod_i C(s_i),
    s_i = sin(pi m_i / N) (alias sum of the kernel; Jing 2005, cited in Sec. 4),
    checked on the mean over all binned modes of several seeds (Eq. 3 shot noise)."""
    n = 32
    ratios = []
    for seed in range(4):
        gal, ran, geo = synth.poisson_cube(4000, 20000, seed=100 + seed)
        nm = oracle.catalog_sums(gal, ran)
        bins = BinSpec(0.0, 0.02, 15)
        res = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, compensate=False,
                                    ell_max=0, return_modes=True)
        bidx, w, _ = mode_bins(n, geo.box_len, bins)
        mx, my, mz, _ = half_modes(n)
        C = (closed(np.sin(np.pi * mx / n)) * closed(np.sin(np.pi * my / n)) *
             closed(np.sin(np.pi * mz / n)))
        A0 = res.modes["A0"]
        sel = bidx >= 0
        r = (np.abs(A0) ** 2 / (nm.S * C))[sel]
        ratios.append(r)
    r = np.concatenate(ratios)
    err = np.std(r) / math.sqrt(r.size)
    assert abs(np.mean(r) - 1.0) < 4 * err


_ALIAS_CACHE = {}


def _alias_sums(kind):
    """Poisson summation of one particle's assignment along each axis, from the
    kernel's analytic transform sinc(w/2)^p alone (none of the oracle's code):

        sum_j W(u - j) e^{-i theta j} = sum_q What(theta + 2 pi q) e^{-i (theta + 2 pi q) u},

    theta = 2 pi m / N over the rfftn labels.  Returns per axis (S, T) with T the
    same sum weighted by (-1)^q, the particle's grid coordinates u and the thetas."""
    if kind in _ALIAS_CACHE:
        return _ALIAS_CACHE[kind]
    n, H = 8, 1.5
    box_min = (-3.25, 10.5, 0.75)
    pos = np.array([[box_min[d] + H * f for d, f in enumerate((2.23, 5.71, 7.38))]], dtype=np.float32)
    u = [(float(pos[0, d]) - box_min[d]) / H for d in range(3)]
    p = {"ngp": 1, "cic": 2, "tsc": 3}[kind]
    Q = 2 ** 20 if kind == "ngp" else 2 ** 16  # NGP's terms fall as 1/q, the others' as 1/q^p
    q = np.arange(-Q, Q + 1)
    sign = np.where(q % 2 == 0, 1.0, -1.0)
    m_xy = np.fft.fftfreq(n, d=1.0 / n)
    thetas = [2 * np.pi * m / n for m in (m_xy, m_xy, np.arange(n // 2 + 1))]
    sums = []
    for d in range(3):
        S, T = [], []
        frac = u[d] - math.floor(u[d])  # e^{-2 pi i q u} only needs u mod 1
        tail = np.exp(-2j * np.pi * q * frac)
        for th in thetas[d]:
            om = th + 2 * np.pi * q
            terms = np.sinc(om / (2 * np.pi)) ** p * tail * np.exp(-1j * th * u[d])
            S.append(np.sum(terms))
            T.append(np.sum(sign * terms))
        sums.append((np.array(S), np.array(T)))
    _ALIAS_CACHE[kind] = (n, H, box_min, pos, sums, thetas, p)
    return _ALIAS_CACHE[kind]


def _outer(a, b, c):
    return a[:, None, None] * b[None, :, None] * c[None, None, :]


@pytest.mark.parametrize("kind,tol", [("ngp", 3e-6), ("cic", 1e-9), ("tsc", 1e-12)])
@pytest.mark.parametrize("interlace", [False, True])
@pytest.mark.parametrize("compensate", [False, True])
def test_single_particle_alias_sum(kind, tol, interlace, compensate):
    """Interlacing and window compensation, exactly (Sec. 4's mesh step): one
    particle of unit net weight (a galaxy of weight 7/4 and a random of weight 1 at
    the same point, alpha = 3/4).  By Poisson summation its mesh transform is
    prod_i S_i, S_i = sum_q What(theta_i + 2 pi q) e^{-i (theta_i + 2 pi q) u_i}.
    The mesh at +H/2 brought back by e^{-i theta.(1,1,1)/2} carries (-1)^(q_x+q_y+q_z)
    on each alias, so the interlaced mean keeps the aliases of even q_x + q_y + q_z:
    (prod S + prod T) / 2.  Compensation divides by prod What(theta_i), leaving the
    exact mode e^{-i k.(x - box_min)} plus the surviving aliases.  A flipped
    interlacing phase or a mesh shifted the other way gives
    (prod S + e^{+-i sum theta} prod T) / 2 instead, which is checked to be far off."""
    n, H, box_min, pos, sums, thetas, p = _alias_sums(kind)
    gal = synth.Catalog.from_positions(pos, 1.75, 1e-3)
    ran = synth.Catalog.from_positions(pos, 1.0, 1e-3)
    geo = synth.Geometry(box_min, n * H, (0.0, 0.0, 0.0))
    res = oracle.fft_multipoles(gal, ran, geo, n, BinSpec(0.0, 0.1, 3), assign=kind, interlace=interlace,
                                compensate=compensate, ell_max=0, alpha=0.75, return_modes=True)
    A0 = res.modes["A0"]
    S = _outer(*(s for s, _ in sums))
    T = _outer(*(t for _, t in sums))
    Wk = _outer(*(np.sinc(th / (2 * np.pi)) ** p for th in thetas)) if compensate else 1.0
    want = (0.5 * (S + T) if interlace else S) / Wk
    scale = np.abs(want).max()
    assert np.abs(A0 - want).max() <= tol * scale
    if interlace:
        sum_th = _outer(*(np.exp(1j * th) for th in thetas))
        for wrong in (sum_th, np.conj(sum_th)):
            assert np.abs(A0 - 0.5 * (S + wrong * T) / Wk).max() > 0.5 * scale
    if compensate:
        # the unaliased mode: at low |m| the compensated value is close to e^{-i k.(x - box_min)}
        u = [(float(pos[0, d]) - box_min[d]) / H for d in range(3)]
        exact = _outer(*(np.exp(-1j * th * u[d]) for d, th in enumerate(thetas)))
        assert abs(A0[1, 0, 0] - exact[1, 0, 0]) < (0.2 if kind == "ngp" else 0.06)


# --------------------------------------------------------------------------
# The three implementations of Sec. 4
# --------------------------------------------------------------------------

def test_three_routes_agree_ngp_on_nodes():
    """Particles on nodes + NGP + no window: the mesh holds the particles exactly, so
    FFT-based, sum-grid and sum-gal agree to rounding (Sec. 4, Fig. 1 structure)."""
    n = 16
    gal, ran, geo = synth.on_node_catalog(n, (64.0, 32.0, 96.0), 128.0, 300, 1500, seed=3)
    bins = BinSpec(0.0, 0.02, 20)
    f = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="ngp", compensate=False)
    g = oracle.sum_gal(gal, ran, geo, n, bins)
    F = oracle.assign_mesh(gal, ran, f.norm.alpha, geo.box_min, geo.box_len, n, "ngp")
    s = oracle.sum_grid([F], gal, ran, geo, n, bins, assign="ngp", compensate=False)
    for name in ("p0", "p2", "p4"):
        assert _rel(getattr(f, name), getattr(g, name)) < 1e-12, name
        assert _rel(getattr(f, name), getattr(s, name)) < 1e-12, name


@pytest.mark.parametrize("kind,interlace", [("cic", False), ("tsc", True), ("ngp", True)])
def test_sum_grid_equals_fft_every_mode(kind, interlace):
    """The 22-FFT decomposition equals the direct (k.r)^n sum over nodes at every
    binned mode (Sec. 3: no further approximation), interlaced and compensated."""
    n = 16
    gal, ran, geo = synth.poisson_cube(400, 2000, side=200.0, center=(150.0, 40.0, -120.0), seed=9)
    bins = BinSpec(0.0, 0.01, 40)
    f = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, interlace=interlace,
                              return_modes=True)
    meshes = [oracle.assign_mesh(gal, ran, f.norm.alpha, geo.box_min, geo.box_len, n, kind, il)
              for il in ([False, True] if interlace else [False])]
    s = oracle.sum_grid(meshes, gal, ran, geo, n, bins, assign=kind)
    bidx, _, _ = mode_bins(n, geo.box_len, bins)
    sel = bidx >= 0
    for key, n_ in (("A0", 0), ("A2", 2), ("A4", 4)):
        a = f.modes[key][sel]
        b = s.modes[n_]
        assert np.max(np.abs(a - b)) / np.max(np.abs(a)) < 1e-11, key
    for name in ("p0", "p2", "p4"):
        assert _rel(getattr(f, name), getattr(s, name)) < 1e-11


def test_legendre_combination_matches_eq4():
    """Eqs. (6)-(8) equal Eq. (4) with the Legendre polynomials evaluated directly."""
    gal, ran, geo = synth.poisson_cube(300, 1500, side=300.0, seed=21)
    bins = BinSpec(0.0, 0.03, 12)
    a = oracle.sum_gal(gal, ran, geo, 12, bins)
    b = oracle.sum_gal(gal, ran, geo, 12, bins, legendre=True)
    for name in ("p0", "p2", "p4"):
        assert _rel(getattr(a, name), getattr(b, name)) < 1e-12


# --------------------------------------------------------------------------
# Limits and symmetries
# --------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_distant_observer_limit(axis):
    """Observer 1e9 Mpc/h away along -axis: every r_hat ~ e_axis, so A_2 -> mu^2 A_0
    and A_4 -> mu^4 A_0 with mu = k_axis/k, and P_2, P_4 reduce to the single-FFT
    plane-parallel estimator."""
    gal, ran, geo = synth.poisson_cube(1500, 7500, side=400.0, center=(0.0, 0.0, 0.0), seed=31)
    far = [0.0, 0.0, 0.0]
    far[axis] = -1.0e9
    geo = synth.Geometry(geo.box_min, geo.box_len, tuple(far))
    n = 16
    bins = BinSpec(0.0, 0.01, 30)
    f = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="cic", return_modes=True)
    mx, my, mz, _ = half_modes(n)
    kk = [mx, my, mz][axis].astype(float)
    k2 = (mx * mx + my * my + mz * mz).astype(float)
    mu2 = np.where(k2 > 0, kk * kk / np.where(k2 > 0, k2, 1), 0)
    A0 = f.modes["A0"]
    bidx, w, _ = mode_bins(n, geo.box_len, bins)
    sel = bidx >= 0
    assert np.max(np.abs(f.modes["A2"] - mu2 * A0)[sel]) < 1e-5 * np.max(np.abs(A0[sel]))
    assert np.max(np.abs(f.modes["A4"] - mu2 ** 2 * A0)[sel]) < 1e-5 * np.max(np.abs(A0[sel]))
    p2 = np.bincount(bidx[sel], (w * (3 * mu2 - 1) * np.abs(A0) ** 2)[sel], bins.n_bins)
    nb = f.n_modes
    with np.errstate(invalid="ignore"):
        p2 = 2.5 / f.norm.I * p2 / nb
    m = np.isfinite(p2)
    assert np.max(np.abs(p2 - f.p2)[m]) < 1e-5 * np.max(np.abs(f.p0[m]))


def test_p0_observer_invariant():
    """A_0 does not involve the LOS (Sec. 2): moving only the observer leaves P_0
    bit-identical while P_2 changes."""
    gal, ran, geo = synth.poisson_cube(800, 4000, side=300.0, seed=41)
    bins = BinSpec(0.0, 0.02, 15)
    a = oracle.fft_multipoles(gal, ran, geo, 16, bins, assign="tsc", interlace=True)
    geo2 = synth.Geometry(geo.box_min, geo.box_len, (123.0, -45.0, 678.0))
    b = oracle.fft_multipoles(gal, ran, geo2, 16, bins, assign="tsc", interlace=True)
    m = np.isfinite(a.p0)
    assert np.array_equal(a.p0[m], b.p0[m])
    assert not np.allclose(a.p2[m], b.p2[m])


def test_translation_and_axis_permutation_invariance():
    """Shifting particles, box and observer together, or relabelling the axes
    (x<->y<->z cyclically, or x<->z), leaves P_l unchanged: catches mis-indexed
    terms of Eqs. (10)-(13)."""
    gal, ran, geo = synth.poisson_cube(800, 4000, side=256.0, center=(300.0, 180.0, 90.0), seed=51)

    def quantise(c):  # multiples of 1/256 stay exact in float32 under the shifts below
        return synth.Catalog.from_positions(np.round(c.positions().astype(np.float64) * 256) / 256,
                                            c.w, c.nbar)

    gal, ran = quantise(gal), quantise(ran)
    bins = BinSpec(0.0, 0.02, 12)
    ref = oracle.fft_multipoles(gal, ran, geo, 16, bins, assign="cic")

    def rebuild(perm, shift):
        def cat(c):
            p = c.positions().astype(np.float64)[:, perm] + shift
            return synth.Catalog.from_positions(p, c.w, c.nbar)
        bm = np.asarray(geo.box_min)[perm] + shift
        ob = np.asarray(geo.observer)[perm] + shift
        return cat(gal), cat(ran), synth.Geometry(tuple(bm), geo.box_len, tuple(ob))

    for perm, shift in [([0, 1, 2], np.array([64.0, -128.0, 32.0])),
                        ([1, 2, 0], np.zeros(3)), ([2, 1, 0], np.zeros(3))]:
        g2, r2, geo2 = rebuild(perm, shift)
        res = oracle.fft_multipoles(g2, r2, geo2, 16, bins, assign="cic")
        for name in ("p0", "p2", "p4"):
            assert _rel(getattr(ref, name), getattr(res, name)) < 1e-9, (perm, name)


def test_field_identities():
    """sum_i B_ii = A_0 and C_ixx + C_iyy + C_izz... (r_x^2 + r_y^2 + r_z^2 = r^2)
    on the transformed fields, and the on-axis reductions A_2 = B_xx, A_4 = C_xxx."""
    gal, ran, geo = synth.poisson_cube(500, 2500, side=200.0, center=(120.0, 80.0, 60.0), seed=61)
    n = 16
    nm = oracle.catalog_sums(gal, ran)
    F = oracle.assign_mesh(gal, ran, nm.alpha, geo.box_min, geo.box_len, n, "cic")
    rx, ry, rz = node_offsets(geo.box_min, geo.box_len, n, geo.observer, False)
    X, Y, Z = rx[:, None, None], ry[None, :, None], rz[None, None, :]
    r2 = X * X + Y * Y + Z * Z

    def ft(name):
        (a, b, c), d = field_monomial(name)
        return np.fft.rfftn(F * X ** a * Y ** b * Z ** c / r2 ** (d // 2))

    A0 = np.fft.rfftn(F)
    assert np.allclose(ft("Bxx") + ft("Byy") + ft("Bzz"), A0, rtol=0, atol=1e-10 * np.abs(A0).max())
    bxx = ft("Bxx")
    assert np.allclose(ft("Cxxx") + ft("Cxyy") + ft("Cxzz"), bxx, atol=1e-10 * np.abs(bxx).max())
    from oracle.estimator import mesh_transforms
    T = mesh_transforms(F, rx, ry, rz, 4, 1)
    for m in range(1, n // 2):
        assert T["A2"][m, 0, 0] == pytest.approx(bxx[m, 0, 0], rel=1e-10, abs=1e-12)
        assert T["A4"][m, 0, 0] == pytest.approx(ft("Cxxx")[m, 0, 0], rel=1e-10, abs=1e-12)


# --------------------------------------------------------------------------
# l = 6 (the same decomposition one order up; Sec. 3)
# --------------------------------------------------------------------------

def test_l6_terms_cover_every_monomial_once():
    assert len(A6_TERMS) == 28
    assert len({kp for _, kp, _ in A6_TERMS}) == 28
    assert sum(c for c, _, _ in A6_TERMS) == 3 ** 6   # (1 + 1 + 1)^6


def test_l6_routes_agree_ngp_on_nodes():
    """Particles on nodes + NGP + no window: the 28-field FFT route, sum-gal with
    mu-powers and sum-gal with L_6 evaluated directly give the same P_6."""
    n = 16
    gal, ran, geo = synth.on_node_catalog(n, (64.0, 32.0, 96.0), 128.0, 300, 1500, seed=3)
    bins = BinSpec(0.0, 0.02, 20)
    f = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="ngp", compensate=False, ell_max=6)
    g = oracle.sum_gal(gal, ran, geo, n, bins, ell_max=6)
    gl = oracle.sum_gal(gal, ran, geo, n, bins, ell_max=6, legendre=True)
    assert _rel(f.p6, g.p6) < 1e-12
    assert _rel(g.p6, gl.p6) < 1e-12
    for name in ("p0", "p2", "p4"):   # adding l = 6 leaves the lower multipoles alone
        assert _rel(getattr(f, name), getattr(g, name)) < 1e-12


def test_l6_distant_observer_limit():
    """Observer far along -z: A_6 -> mu^6 A_0 with mu = k_z/k at every mode."""
    gal, ran, geo = synth.poisson_cube(1500, 7500, side=400.0, center=(0.0, 0.0, 0.0), seed=32)
    geo = synth.Geometry(geo.box_min, geo.box_len, (0.0, 0.0, -1.0e9))
    n = 16
    bins = BinSpec(0.0, 0.01, 30)
    f = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="cic", ell_max=6, return_modes=True)
    mx, my, mz, _ = half_modes(n)
    k2 = (mx * mx + my * my + mz * mz).astype(float)
    mu2 = np.where(k2 > 0, mz * mz / np.where(k2 > 0, k2, 1), 0)
    A0 = f.modes["A0"]
    bidx, _, _ = mode_bins(n, geo.box_len, bins)
    sel = bidx >= 0
    assert np.max(np.abs(f.modes["A6"] - mu2 ** 3 * A0)[sel]) < 1e-5 * np.max(np.abs(A0[sel]))
