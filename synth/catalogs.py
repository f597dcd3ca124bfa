"""Seeded synthetic galaxy and random catalogues.

Every generator takes an explicit seed and uses numpy's PCG64 stream, so the same
call gives the same float32 arrays on every machine.  Positions are comoving
Cartesian coordinates in Mpc/h with the observer at ``Geometry.observer``.

The workloads mirror the survey shapes of the paper (Sec. 4: a 3500 Mpc/h box,
alpha^-1 ~ 10, CIC assignment) and the synthetic stand-ins for them:

* ``poisson_cube``   -- unclustered points in a cube (the 32^3 CIC small case and
                        the batched-mock catalogues).
* ``poisson_shell``  -- unclustered points in a full-sky shell clipped to a cube
                        centred on the observer (the 512^3 survey-shaped case).
* ``zeldovich_cone`` -- a clustered redshift-space mock: a displaced lattice
                        (Zel'dovich moves of a seeded Gaussian field) with a radial
                        redshift-space shift, selected in a cone with a Gaussian
                        radial distribution; FKP weights.
* ``zeldovich_cube`` -- the same clustered construction inside a cube.
* ``on_node_catalog``-- points placed exactly on mesh nodes (exactness checks).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Catalog:
    """Structure-of-arrays catalogue; all arrays float32 of length n."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    w: np.ndarray
    nbar: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def positions(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)

    @staticmethod
    def from_positions(pos: np.ndarray, w, nbar) -> "Catalog":
        pos = np.asarray(pos, dtype=np.float32)
        n = pos.shape[0]
        w = np.broadcast_to(np.asarray(w, dtype=np.float32), (n,)).copy()
        nbar = np.broadcast_to(np.asarray(nbar, dtype=np.float32), (n,)).copy()
        return Catalog(np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
                       np.ascontiguousarray(pos[:, 2]), w, nbar)


@dataclasses.dataclass
class Geometry:
    """Cubic analysis box [box_min, box_min + box_len)^3 and the observer position."""
    box_min: tuple
    box_len: float
    observer: tuple = (0.0, 0.0, 0.0)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Unclustered catalogues
# ---------------------------------------------------------------------------

def poisson_cube(n_gal: int, n_ran: int, side: float = 500.0,
                 center=(600.0, 600.0, 600.0), seed: int = 1,
                 observer=(0.0, 0.0, 0.0)):
    """Uniform galaxies and randoms in the cube ``center +- side/2``; unit weights.

    The analysis box is the cube itself.  nbar is the galaxy number density
    n_gal / side^3 for both catalogues.
    """
    rng = _rng(seed)
    lo = np.asarray(center, dtype=np.float64) - 0.5 * side
    nbar = n_gal / side ** 3

    def draw(n):
        p = lo + side * rng.random((n, 3))
        p = p.astype(np.float32)
        # float32 rounding may land on the upper face; fold it back inside.
        hi = (lo + side).astype(np.float32)
        p = np.where(p >= hi, np.nextafter(hi, np.float32(-np.inf)), p)
        return p

    gal = Catalog.from_positions(draw(n_gal), 1.0, nbar)
    ran = Catalog.from_positions(draw(n_ran), 1.0, nbar)
    geo = Geometry(tuple(float(v) for v in lo), float(side), tuple(float(v) for v in observer))
    return gal, ran, geo


def poisson_shell(n_gal: int, n_ran: int, r_min: float = 600.0, r_max: float = 2000.0,
                  box_len: float = 3500.0, margin: float = 3 * 3500.0 / 512, seed_gal: int = 4,
                  seed_ran: int = 5, chunk: int = 8_000_000):
    """Uniform points in the shell r_min <= r < r_max clipped to the cube of side
    ``box_len`` centred on the observer (origin), kept ``margin`` inside its faces.

    nbar = n_gal / V where V is the clipped-shell volume estimated from the
    acceptance ratio of the random draw (tens of millions of proposals).
    """
    half = 0.5 * box_len - margin
    shell_vol = 4.0 / 3.0 * math.pi * (r_max ** 3 - r_min ** 3)
    proposals = [0]

    def draw(n, seed):
        rng = _rng(seed)
        out = []
        have = 0
        while have < n:
            m = chunk
            u = rng.random(m)
            r = np.cbrt(r_min ** 3 + u * (r_max ** 3 - r_min ** 3))
            d = rng.standard_normal((m, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            p = (d * r[:, None]).astype(np.float32)
            ok = np.all(np.abs(p) < np.float32(half), axis=1)
            proposals[0] += m
            p = p[ok]
            out.append(p)
            have += p.shape[0]
        p = np.concatenate(out)
        accepted_total = p.shape[0]
        return p[:n], accepted_total

    pg, acc_g = draw(n_gal, seed_gal)
    props_g = proposals[0]
    pr, _ = draw(n_ran, seed_ran)
    vol = shell_vol * acc_g / props_g
    nbar = n_gal / vol
    gal = Catalog.from_positions(pg, 1.0, nbar)
    ran = Catalog.from_positions(pr, 1.0, nbar)
    geo = Geometry((-0.5 * box_len,) * 3, float(box_len), (0.0, 0.0, 0.0))
    return gal, ran, geo


def on_node_catalog(n_mesh: int, box_min, box_len: float, n_gal: int, n_ran: int,
                    seed: int = 7, weights: bool = True, observer=(0.0, 0.0, 0.0)):
    """Galaxies and randoms placed exactly on mesh nodes box_min + i*H.

    box_min and H = box_len/n_mesh should be exactly representable (powers of two)
    so that the float32 positions are the node positions.  Weights are drawn from
    [0.5, 1.5) when ``weights`` is set, else 1.
    """
    rng = _rng(seed)
    H = box_len / n_mesh
    lo = np.asarray(box_min, dtype=np.float64)

    def draw(n):
        idx = rng.integers(0, n_mesh, size=(n, 3))
        p = lo + idx * H
        w = (0.5 + rng.random(n)) if weights else np.ones(n)
        return p.astype(np.float32), w.astype(np.float32)

    pg, wg = draw(n_gal)
    pr, wr = draw(n_ran)
    nbar = n_gal / box_len ** 3
    gal = Catalog.from_positions(pg, wg, nbar)
    ran = Catalog.from_positions(pr, wr, nbar)
    return gal, ran, Geometry(tuple(float(v) for v in lo), float(box_len),
                              tuple(float(v) for v in observer))


# ---------------------------------------------------------------------------
# Clustered redshift-space mocks (Zel'dovich displacements + radial RSD)
# ---------------------------------------------------------------------------

def linear_power(k, amp=2.0e4, k0=0.02, slope=-1.5, kcut=0.5):
    """Input power spectrum P(k) = amp (k/k0)^slope exp(-(k/kcut)^2), (Mpc/h)^3."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    nz = k > 0
    out[nz] = amp * (k[nz] / k0) ** slope * np.exp(-(k[nz] / kcut) ** 2)
    return out


def _displacement(n_grid: int, cell: float, rng: np.random.Generator):
    """Zel'dovich displacement field psi (3, n, n, n) of a seeded Gaussian density
    field with the power spectrum ``linear_power`` on a periodic grid."""
    white = rng.standard_normal((n_grid,) * 3)
    wk = np.fft.rfftn(white)
    kf = 2 * np.pi / (n_grid * cell)
    kx = np.fft.fftfreq(n_grid, d=1.0 / n_grid) * kf
    kz = np.fft.rfftfreq(n_grid, d=1.0 / n_grid) * kf
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    amp = np.sqrt(linear_power(np.sqrt(k2)) / cell ** 3)
    dk = wk * amp
    k2[0, 0, 0] = 1.0
    psi = []
    for K in (KX, KY, KZ):
        psi.append(np.fft.irfftn(1j * K * dk / k2, s=(n_grid,) * 3, axes=(0, 1, 2)))
    return np.stack(psi)


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _truncated_gaussian_radii(rng, n, mean, sigma, lo, hi):
    out = []
    have = 0
    while have < n:
        r = rng.normal(mean, sigma, size=2 * (n - have) + 1024)
        r = r[(r >= lo) & (r < hi)]
        out.append(r)
        have += r.shape[0]
    return np.concatenate(out)[:n]


def zeldovich_cone(n_gal: int = 1_000_000, n_ran: int = 5_000_000, n_mesh: int = 256,
                   half_angle_deg: float = 30.0, axis=(1.0, 1.0, 1.0),
                   r_mean: float = 1200.0, r_sigma: float = 300.0, r_lo: float = 300.0,
                   r_hi: float = 2100.0, f_growth: float = 0.7, p_fkp: float = 1.0e4,
                   n_lattice: int = 320, field_len: float = 2048.0, seed_field: int = 2,
                   seed_ran: int = 3, margin_cells: int = 3, origin: float = -64.0, box_len=None):
    """Clustered redshift-space mock in a cone (full opening 2*half_angle_deg).

    Galaxies: a cubic lattice of n_lattice^3 sites over [origin, origin + field_len)^3 is
    displaced by Zel'dovich moves psi, then shifted along the line of sight by
    f (psi . r_hat) r_hat; sites in the cone are kept with probability proportional
    to G(r)/r^2 (G a Gaussian of mean r_mean, width r_sigma truncated to
    [r_lo, r_hi)), then exactly n_gal are drawn without replacement.
    Randoms: radii from G, directions uniform in the cone.
    nbar(r) = n_gal G(r) / (Omega r^2 int G); FKP weights w = 1/(1 + nbar p_fkp).
    The analysis box is the bounding cube of all points plus margin_cells cells, or,
    with box_len given, the cube of that side centred on the points' bounding box.
    """
    rng = _rng(seed_field)
    cell = field_len / n_lattice
    psi = _displacement(n_lattice, cell, rng).astype(np.float32)
    g1 = origin + cell * np.arange(n_lattice, dtype=np.float64)
    ax = _unit(axis)
    cos_t = math.cos(math.radians(half_angle_deg))
    omega = 2 * math.pi * (1 - cos_t)
    gnorm = r_sigma * math.sqrt(2 * math.pi) * 0.5 * (
        math.erf((r_hi - r_mean) / (math.sqrt(2) * r_sigma)) -
        math.erf((r_lo - r_mean) / (math.sqrt(2) * r_sigma)))

    def gauss(r):
        return np.exp(-0.5 * ((r - r_mean) / r_sigma) ** 2)

    # acceptance normaliser: max of G(r)/r^2 on [r_lo, r_hi)
    rr = np.linspace(r_lo, r_hi, 20001)
    amax = float(np.max(gauss(rr) / rr ** 2))

    sel = []
    for i in range(n_lattice):  # one lattice plane at a time bounds the memory
        qx = np.full((n_lattice, n_lattice), g1[i])
        qy, qz = np.meshgrid(g1, g1, indexing="ij")
        x = np.stack([qx + psi[0, i], qy + psi[1, i], qz + psi[2, i]], axis=-1).reshape(-1, 3)
        p = psi[:, i].reshape(3, -1).T
        r = np.linalg.norm(x, axis=1)
        rhat = x / np.maximum(r, 1e-30)[:, None]
        s = x + f_growth * np.sum(p * rhat, axis=1)[:, None] * rhat
        rs = np.linalg.norm(s, axis=1)
        inside = (rs >= r_lo) & (rs < r_hi) & (s @ ax >= cos_t * rs)
        s = s[inside]
        rs = rs[inside]
        keep = rng.random(s.shape[0]) < gauss(rs) / rs ** 2 / amax
        sel.append(s[keep])
    gal_pos = np.concatenate(sel)
    if gal_pos.shape[0] < n_gal:
        raise ValueError(f"lattice too coarse: {gal_pos.shape[0]} < {n_gal} candidates")
    gal_pos = gal_pos[rng.choice(gal_pos.shape[0], size=n_gal, replace=False)]

    rng_r = _rng(seed_ran)
    r = _truncated_gaussian_radii(rng_r, n_ran, r_mean, r_sigma, r_lo, r_hi)
    ct = cos_t + (1 - cos_t) * rng_r.random(n_ran)
    st = np.sqrt(np.maximum(0.0, 1 - ct ** 2))
    ph = 2 * math.pi * rng_r.random(n_ran)
    # orthonormal frame around the cone axis
    e1 = _unit(np.cross(ax, [1.0, 0.0, 0.0] if abs(ax[0]) < 0.9 else [0.0, 1.0, 0.0]))
    e2 = np.cross(ax, e1)
    d = (ct[:, None] * ax + (st * np.cos(ph))[:, None] * e1 + (st * np.sin(ph))[:, None] * e2)
    ran_pos = d * r[:, None]

    def nbar_of(pos):
        rr_ = np.linalg.norm(pos, axis=1)
        return n_gal * gauss(rr_) / (omega * rr_ ** 2 * gnorm)

    nb_g = nbar_of(gal_pos)
    nb_r = nbar_of(ran_pos)
    gal = Catalog.from_positions(gal_pos, 1.0 / (1.0 + nb_g * p_fkp), nb_g)
    ran = Catalog.from_positions(ran_pos, 1.0 / (1.0 + nb_r * p_fkp), nb_r)

    allpos = np.concatenate([gal.positions(), ran.positions()]).astype(np.float64)
    lo = allpos.min(axis=0)
    hi = allpos.max(axis=0)
    if box_len is None:
        ext = float(np.max(hi - lo))
        box_len = ext * n_mesh / (n_mesh - 2 * margin_cells)
        H = box_len / n_mesh
        box_min = tuple(float(v) for v in (lo - margin_cells * H))
    else:
        if float(np.max(hi - lo)) >= box_len:
            raise ValueError("the points do not fit a box of side box_len")
        box_min = tuple(float(v) for v in (0.5 * (lo + hi) - 0.5 * box_len))
    return gal, ran, Geometry(box_min, float(box_len), (0.0, 0.0, 0.0))


def paper_cap(n_gal: int = 525_000, n_ran: int = 5_250_000, seed_field: int = 6, seed_ran: int = 7):
    """Stand-in for the paper's workload (Sec. 4: one survey-shaped mock of ~525 000
    galaxies with ten times as many randoms in a box of side 3500 Mpc/h): clustered
    redshift-space galaxies in a cap of 7000 deg^2 (half-angle 48.7 deg about +z)
    between comoving 1100 and 1900 Mpc/h (n(r) Gaussian about 1500, width 200), FKP
    weights with P_0 = 2e4, in a 3500 Mpc/h box centred on the cap's bounding box."""
    half = math.degrees(math.acos(1.0 - 7000.0 * (math.pi / 180.0) ** 2 / (2.0 * math.pi)))
    return zeldovich_cone(n_gal, n_ran, n_mesh=512, half_angle_deg=half, axis=(0.0, 0.0, 1.0),
                          r_mean=1500.0, r_sigma=200.0, r_lo=1100.0, r_hi=1900.0, p_fkp=2.0e4,
                          n_lattice=400, field_len=3500.0, origin=-1500.0, seed_field=seed_field,
                          seed_ran=seed_ran, box_len=3500.0)


def zeldovich_cube(n_gal: int, n_ran: int, side: float = 500.0, center=(600.0, 600.0, 600.0),
                   f_growth: float = 0.7, n_lattice: int = 128, seed: int = 10,
                   observer=(0.0, 0.0, 0.0)):
    """Clustered redshift-space galaxies in a cube (the cube is the periodic analysis
    box): a displaced lattice with radial RSD, wrapped into the cube, subsampled to
    n_gal; uniform randoms; unit weights; nbar = n_gal/side^3."""
    rng = _rng(seed)
    cell = side / n_lattice
    if n_lattice ** 3 < n_gal:
        raise ValueError("n_lattice^3 must be >= n_gal")
    psi = _displacement(n_lattice, cell, rng).reshape(3, -1).T
    lo = np.asarray(center, dtype=np.float64) - 0.5 * side
    g1 = np.arange(n_lattice, dtype=np.float64) * cell
    qx, qy, qz = np.meshgrid(g1, g1, g1, indexing="ij")
    q = np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1) + lo
    pick = rng.choice(q.shape[0], size=n_gal, replace=False)
    x = q[pick] + psi[pick]
    obs = np.asarray(observer, dtype=np.float64)
    rel = x - obs
    rhat = rel / np.linalg.norm(rel, axis=1, keepdims=True)
    s = x + f_growth * np.sum(psi[pick] * rhat, axis=1)[:, None] * rhat
    s = lo + np.mod(s - lo, side)
    nbar = n_gal / side ** 3
    gpos = s.astype(np.float32)
    hi = (lo + side).astype(np.float32)
    gpos = np.where(gpos >= hi, np.nextafter(hi, np.float32(-np.inf)), gpos)
    rpos = (lo + side * rng.random((n_ran, 3))).astype(np.float32)
    rpos = np.where(rpos >= hi, np.nextafter(hi, np.float32(-np.inf)), rpos)
    gal = Catalog.from_positions(gpos, 1.0, nbar)
    ran = Catalog.from_positions(rpos, 1.0, nbar)
    return gal, ran, Geometry(tuple(float(v) for v in lo), float(side),
                              tuple(float(v) for v in observer))


def batched_cube_specs(n_cat: int = 256, first_seed: int = 1000, meshes=(128, 192, 256),
                       n_gal_range=(200_000, 2_000_000), ran_factor: int = 5):
    """Per-catalogue (seed, n_gal, n_ran, n_mesh) for the batched-mock workload."""
    specs = []
    for i in range(n_cat):
        seed = first_seed + i
        rng = _rng(seed + 7_000_000)
        n_gal = int(rng.integers(n_gal_range[0], n_gal_range[1] + 1))
        mesh = int(meshes[int(rng.integers(0, len(meshes)))])
        specs.append((seed, n_gal, ran_factor * n_gal, mesh))
    return specs


# ---------------------------------------------------------------------------
# Named workloads (estimator settings included)
# ---------------------------------------------------------------------------

def workload(name: str, scale: float = 1.0):
    """Return (gal, ran, geometry, settings) for a named workload.

    settings: dict(n_mesh, assign, interlace, ell_max, k_min, dk, n_bins_to) where
    n_bins_to is the upper k edge (None = Nyquist).  ``scale`` < 1 shrinks particle
    counts (and nothing else) for quick runs.
    """
    if name == "cube32_cic":
        gal, ran, geo = poisson_cube(int(2000 * scale) or 1, int(10000 * scale) or 1, seed=1)
        return gal, ran, geo, dict(n_mesh=32, assign="cic", interlace=False, ell_max=4,
                                   k_min=0.0, dk=0.01, k_max=None)
    if name == "cone256_tsc_il":
        gal, ran, geo = zeldovich_cone(int(1_000_000 * scale), int(5_000_000 * scale))
        return gal, ran, geo, dict(n_mesh=256, assign="tsc", interlace=True, ell_max=4,
                                   k_min=0.0, dk=0.01, k_max=None)
    if name in ("paper512_cic", "paper1024_cic"):
        # the same mock on the two meshes of the paper's timing table (Table 1)
        gal, ran, geo = paper_cap(int(525_000 * scale), int(5_250_000 * scale))
        return gal, ran, geo, dict(n_mesh=512 if name == "paper512_cic" else 1024, assign="cic",
                                   interlace=False, ell_max=4, k_min=0.0, dk=0.01, k_max=None)
    if name == "shell512_tsc_il":
        gal, ran, geo = poisson_shell(int(10_000_000 * scale), int(50_000_000 * scale))
        return gal, ran, geo, dict(n_mesh=512, assign="tsc", interlace=True, ell_max=4,
                                   k_min=0.0, dk=0.01, k_max=0.4)
    raise KeyError(name)
