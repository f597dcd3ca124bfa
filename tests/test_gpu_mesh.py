"""The assigned mesh F of Eq. 1, node by node, read back through ys_plan_copy_mesh.

Against the FP64 oracle deposit: |F_gpu - F_oracle| <= 2e-6 A + 1e-6 max(A) at every
node, A being the same deposit of |w| (the sum of the magnitudes that meet at the
node).  The float side rounds each weight product and locates each particle to about
1e-7 of a cell, so its error per contribution is a few 1e-7 |w|; a particle on the
wrong node, a dropped or doubled stencil weight, or a wrong sign moves a node by a
whole contribution.  The mesh total equals sum w_gal - alpha sum w_ran (every stencil
sums to one).

The sorted assignment sums nodes exactly in fixed point, so its mesh must not depend
on the order of the particles: a permuted catalogue gives the same mesh bit for bit.
A crowded tile (over a million records) adds its coarser fixed-point budget to the
bar; a tile holding a NaN weight is summed in float, and the NaN reaches exactly the
nodes of its stencil.
"""
import numpy as np
import pytest

import synth
from oracle.assignment import assign_mesh
from oracle.normalization import catalog_sums
from synth.catalogs import Catalog

torch = pytest.importorskip("torch")
ys = pytest.importorskip("paper_1505_05341_gb300")

pytestmark = pytest.mark.gpu


def to_dev(cat):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cat.x, cat.y, cat.z, cat.w, cat.nbar))


def gpu_mesh(gal, ran, geo, n, kind, interlace):
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign=kind, interlace=interlace, dk=0.05,
                 n_bins=4, stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.assign(to_dev(gal), to_dev(ran))
        return plan.mesh()


def oracle_meshes(gal, ran, geo, n, kind, interlace):
    alpha = catalog_sums(gal, ran).alpha
    absg = Catalog(gal.x, gal.y, gal.z, np.abs(gal.w), gal.nbar)
    absr = Catalog(ran.x, ran.y, ran.z, np.abs(ran.w), ran.nbar)
    refs, bounds = [], []
    for shift in ([False, True] if interlace else [False]):
        refs.append(assign_mesh(gal, ran, alpha, geo.box_min, geo.box_len, n, kind, interlaced=shift))
        bounds.append(assign_mesh(absg, absr, -abs(alpha), geo.box_min, geo.box_len, n, kind, interlaced=shift))
    return np.stack(refs), np.stack(bounds), alpha


def check_mesh(got, gal, ran, geo, n, kind, interlace, label, extra=0.0):
    ref, bound, alpha = oracle_meshes(gal, ran, geo, n, kind, interlace)
    assert got.shape == ref.shape
    err = np.abs(got.astype(np.float64) - ref)
    tol = 2e-6 * bound + 1e-6 * bound.max() + extra
    worst = float(np.max(err / tol))
    print(f"{label}: worst node error / tolerance {worst:.3g}, max |F| {np.abs(ref).max():.3g}")
    assert worst <= 1.0, (label, np.unravel_index(np.argmax(err / tol), err.shape))
    total = float(np.sum(gal.w, dtype=np.float64) - alpha * np.sum(ran.w, dtype=np.float64))
    scale = float(np.sum(np.abs(gal.w), dtype=np.float64) + abs(alpha) * np.sum(np.abs(ran.w), dtype=np.float64))
    for j in range(got.shape[0]):
        assert abs(float(np.sum(got[j], dtype=np.float64)) - total) <= 1e-6 * scale, (label, j)


@pytest.mark.parametrize("n,kind,interlace", [(32, "ngp", False), (64, "cic", True), (64, "tsc", True),
                                              (96, "tsc", False)])
def test_mesh_matches_oracle(n, kind, interlace):
    gal, ran, geo = synth.zeldovich_cube(40_000, 200_000, seed=31)
    got = gpu_mesh(gal, ran, geo, n, kind, interlace)
    check_mesh(got, gal, ran, geo, n, kind, interlace, f"{n}_{kind}_{interlace}")


def test_mesh_with_weights_and_nodes():
    """Uneven positive weights, and particles placed on nodes and cell edges."""
    n = 32
    gal, ran, geo = synth.on_node_catalog(n, (0.0, 0.0, 0.0), 320.0, 3_000, 12_000, seed=5)
    rng = np.random.default_rng(8)
    gal.w[:] = rng.uniform(0.2, 3.0, gal.n).astype(np.float32)
    ran.w[:] = rng.uniform(0.5, 1.5, ran.n).astype(np.float32)
    for kind in ("ngp", "cic", "tsc"):
        got = gpu_mesh(gal, ran, geo, n, kind, True)
        check_mesh(got, gal, ran, geo, n, kind, True, f"nodes_{kind}")


def test_mesh_independent_of_particle_order():
    gal, ran, geo = synth.zeldovich_cube(50_000, 250_000, seed=44)
    rng = np.random.default_rng(3)

    def permuted(c):
        p = rng.permutation(c.n)
        return Catalog(*(np.ascontiguousarray(a[p]) for a in (c.x, c.y, c.z, c.w, c.nbar)))

    for kind, interlace in (("tsc", True), ("cic", False)):
        a = gpu_mesh(gal, ran, geo, 64, kind, interlace)
        b = gpu_mesh(permuted(gal), permuted(ran), geo, 64, kind, interlace)
        c = gpu_mesh(gal, ran, geo, 64, kind, interlace)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), kind
        assert np.array_equal(a.view(np.uint32), c.view(np.uint32)), kind


def test_crowded_tile():
    """1.2e6 galaxies in a ball of two cells' radius, all in one tile: ~1.25e6 records,
    ~3e5 contributions at the densest nodes.  With that many records and |w| up to 6
    (alpha = 6) the tile's fixed-point scale is 2^-17 (s = floor(30 + sb - log2(n w_m)),
    sb = floor(31 - log2 n) = 10), so each stencil weight may move by 2^-18 and the
    many TSC tail weights below that round mostly to zero.  The bar adds that budget,
    K 2^-16 (K: particles within two cells of the node on every axis, a superset of
    those whose stencil reaches it; two bits of margin) to the usual one.  Float sums
    drop every weight below half an ulp of these nodes: ~1e-3 relative, 30 times more."""
    n, side = 32, 320.0
    rng = np.random.default_rng(21)
    m = 1_200_000
    centre = np.array([70.0, 90.0, 150.0])
    d = rng.normal(size=(m, 3))
    d *= (rng.uniform(size=(m, 1)) ** (1 / 3) * 20.0) / np.linalg.norm(d, axis=1, keepdims=True)
    gpos = (centre + d).astype(np.float32)
    rpos = rng.uniform(0.0, side, size=(200_000, 3)).astype(np.float32)
    gal = Catalog.from_positions(gpos, np.ones(m, np.float32), np.full(m, 1e-4, np.float32))
    ran = Catalog.from_positions(rpos, np.ones(len(rpos), np.float32), np.full(len(rpos), 1e-4, np.float32))
    geo = synth.catalogs.Geometry((0.0, 0.0, 0.0), side, (-50.0, -50.0, -50.0))
    got = gpu_mesh(gal, ran, geo, n, "tsc", True)
    cells = np.floor(np.concatenate([gpos, rpos]).astype(np.float64) / (side / n)).astype(int) % n
    hist = np.zeros((n, n, n))
    np.add.at(hist, (cells[:, 0], cells[:, 1], cells[:, 2]), 1.0)
    k_near = np.zeros_like(hist)
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            for dz in range(-2, 3):
                k_near += np.roll(hist, (dx, dy, dz), axis=(0, 1, 2))
    check_mesh(got, gal, ran, geo, n, "tsc", True, "crowded", extra=k_near * 2.0 ** -16)


def test_nan_weight_reaches_only_its_nodes():
    """A tile holding a non-finite weight is summed in float: with alpha fixed, one
    NaN-weighted galaxy makes exactly the nodes of its stencil NaN (as in the FP64
    oracle), and every other node of that tile still matches."""
    gal, ran, geo = synth.zeldovich_cube(20_000, 100_000, seed=12)
    gal.w[123] = np.nan
    n, alpha = 64, 0.2
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, dk=0.05, n_bins=4,
                 alpha=alpha, stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.assign(to_dev(gal), to_dev(ran))
        got = plan.mesh()
    ref = np.stack([assign_mesh(gal, ran, alpha, geo.box_min, geo.box_len, n, "tsc", interlaced=s)
                    for s in (False, True)])
    nan = np.isnan(ref)
    assert 0 < nan.sum() <= 2 * 27
    assert np.array_equal(np.isnan(got), nan)
    absg = Catalog(gal.x, gal.y, gal.z, np.nan_to_num(np.abs(gal.w)), gal.nbar)
    bound = np.stack([assign_mesh(absg, ran, -alpha, geo.box_min, geo.box_len, n, "tsc", interlaced=s)
                      for s in (False, True)])
    err = np.abs(got[~nan].astype(np.float64) - ref[~nan])
    assert np.all(err <= 2e-6 * bound[~nan] + 1e-6 * bound.max())


def test_copy_mesh_before_assignment_is_state_error():
    with ys.Plan(32, (0.0, 0.0, 0.0), 100.0, dk=0.05, n_bins=4) as plan:
        with pytest.raises(ys.YstatError) as ei:
            plan.mesh()
        assert ei.value.status == ys.ystat.YS_ERR_STATE
