"""GPU path (through the C ABI) against the FP64 oracle, shell by shell.

Tolerance: for every multipole l, in every shell where |P_l| > 1e-2 * P_raw
(P_raw = <|A_0|^2>/I, the monopole before the shot noise is subtracted: after the
subtraction P_0 of an unclustered catalogue crosses zero, and a threshold tied to it
would select noise), |P_l^gpu - P_l^oracle| <= 1e-4 |P_l^oracle|.  Mode counts are exact and
the mean |k| agrees to 1e-12.  The worst relative error per shell is printed.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.binning import BinSpec

torch = pytest.importorskip("torch")
ys = pytest.importorskip("paper_1505_05341_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-4


def to_dev(cat):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cat.x, cat.y, cat.z, cat.w, cat.nbar))


def run_gpu(gal, ran, geo, n, bins, assign="cic", interlace=False, ell=4, compensate=True, alpha=-1.0):
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign=assign, interlace=interlace,
                 compensate=compensate, ell_max=ell, k_min=bins.k_min, dk=bins.dk, n_bins=bins.n_bins,
                 alpha=alpha, stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.assign(to_dev(gal), to_dev(ran))
        return plan.measure()


def compare(res, ref, ell, label=""):
    nm = ref.n_modes
    assert np.array_equal(res.n_modes, nm), label
    has = nm > 0
    np.testing.assert_allclose(res.k[has], ref.k[has], rtol=1e-12)
    assert np.all(np.isnan(res.p0[~has]))
    assert res.alpha == pytest.approx(ref.norm.alpha, rel=1e-7)
    assert res.norm_I == pytest.approx(ref.norm.I, rel=1e-6)
    raw = np.where(has, ref.sum0 / np.where(has, nm, 1) / ref.norm.I, 0.0)
    worst = {}
    for l in (0, 2, 4):
        if l > ell:
            assert np.all(np.isnan(getattr(res, f"p{l}")))
            continue
        g, o = getattr(res, f"p{l}"), getattr(ref, f"p{l}")
        sel = has & (np.abs(o) > 1e-2 * raw)
        rel = np.abs(g[sel] - o[sel]) / np.abs(o[sel])
        worst[l] = float(rel.max()) if rel.size else 0.0
        assert sel.sum() > 0 or l > 0, label
        if rel.size:
            assert rel.max() <= TOL, (label, l, rel.max(), np.nonzero(sel)[0][np.argmax(rel)])
    print(f"{label}: worst rel err per multipole {worst}")
    return worst


def test_cube32_cic_small_case():
    """2000 Poisson galaxies + 10000 randoms, 500 Mpc/h cube, 32^3 CIC, l <= 4,
    shells of 0.01 h/Mpc up to Nyquist."""
    gal, ran, geo, s = synth.workload("cube32_cic")
    bins = BinSpec.up_to(np.pi * 32 / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, 32, bins, assign="cic")
    res = run_gpu(gal, ran, geo, 32, bins, "cic")
    compare(res, ref, 4, "cube32_cic")
    assert res.shot_noise == pytest.approx(75000.0, rel=1e-6)


def test_ngp_on_nodes_matches_direct_sum():
    """Particles on nodes + NGP + no window: GPU = oracle FFT = oracle sum-gal."""
    n = 16
    gal, ran, geo = synth.on_node_catalog(n, (64.0, 32.0, 96.0), 128.0, 300, 1500, seed=3)
    bins = BinSpec(0.0, 0.02, 20)
    ref = oracle.sum_gal(gal, ran, geo, n, bins)
    res = run_gpu(gal, ran, geo, n, bins, "ngp", compensate=False)
    compare(res, ref, 4, "ngp_on_nodes")


@pytest.mark.parametrize("n,kind,interlace,ell", [
    (64, "tsc", True, 4),
    (96, "cic", False, 2),
    (128, "tsc", False, 0),
    (192, "cic", True, 4),
    (32, "ngp", True, 4),
])
def test_observer_centred_box(n, kind, interlace, ell):
    """Box centred on the observer (the observer sits on a mesh node; every octant of
    LOS directions), several tiles per axis and ragged pencil blocks."""
    gal, ran, geo = synth.poisson_cube(20_000, 100_000, side=1000.0, center=(0.0, 0.0, 0.0), seed=n)
    bins = BinSpec.up_to(0.9 * np.pi * n / geo.box_len, 0.007)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, interlace=interlace, ell_max=ell)
    res = run_gpu(gal, ran, geo, n, bins, kind, interlace, ell)
    compare(res, ref, ell, f"centred_{n}_{kind}_{interlace}_{ell}")


def test_clustered_cube_tsc_interlaced():
    """Clustered redshift-space galaxies (Zel'dovich + radial RSD), 128^3 TSC
    interlaced: P_2 and P_4 carry signal."""
    gal, ran, geo = synth.zeldovich_cube(150_000, 750_000, seed=12)
    bins = BinSpec.up_to(np.pi * 128 / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, 128, bins, assign="tsc", interlace=True)
    res = run_gpu(gal, ran, geo, 128, bins, "tsc", True)
    compare(res, ref, 4, "zeldovich_cube128")


def test_cone_mock_256_tsc_interlaced():
    """The clustered cone mock: 1e6 galaxies + 5e6 randoms, FKP weights, 256^3 TSC
    with interlacing, l <= 4, shells of 0.01 h/Mpc up to Nyquist."""
    gal, ran, geo, s = synth.workload("cone256_tsc_il")
    bins = BinSpec.up_to(np.pi * 256 / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, 256, bins, assign="tsc", interlace=True)
    res = run_gpu(gal, ran, geo, 256, bins, "tsc", True)
    compare(res, ref, 4, "cone256")


def test_outside_box_reported():
    gal, ran, geo = synth.poisson_cube(100, 500, seed=2)
    gal.x[0] = geo.box_min[0] - 10.0
    bins = BinSpec(0.0, 0.02, 5)
    with ys.Plan(16, geo.box_min, geo.box_len, geo.observer, n_bins=bins.n_bins, dk=bins.dk) as plan:
        plan.assign(to_dev(gal), to_dev(ran))
        with pytest.raises(ys.YstatError):
            plan.measure()
        r = plan.measure(allow_outside=True)
        assert r.status == ys.ystat.YS_ERR_ARG


def test_measure_before_assign_is_state_error():
    with ys.Plan(16, (0.0, 0.0, 0.0), 100.0) as plan:
        with pytest.raises(ys.YstatError) as ei:
            plan.measure()
        assert ei.value.status == ys.ystat.YS_ERR_STATE


def test_empty_galaxy_catalogue():
    """No galaxies, alpha given: F = -alpha * randoms; the path still runs and
    matches the oracle (the shot noise is then alpha^2 sum w^2 / I)."""
    gal, ran, geo = synth.poisson_cube(1, 5000, seed=4)
    gal = synth.Catalog(gal.x[:0], gal.y[:0], gal.z[:0], gal.w[:0], gal.nbar[:0])
    bins = BinSpec(0.0, 0.02, 5)
    ref = oracle.fft_multipoles(gal, ran, geo, 16, bins, alpha=0.2)
    res = run_gpu(gal, ran, geo, 16, bins, alpha=0.2)
    compare(res, ref, 4, "empty_galaxies")


def test_host_entry_point_matches_oracle():
    """ys_estimate_host (host arrays, copies inside) meets the same bar."""
    gal, ran, geo, s = synth.workload("cube32_cic")
    bins = BinSpec.up_to(np.pi * 32 / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, 32, bins, assign="cic")
    with ys.Plan(32, geo.box_min, geo.box_len, geo.observer, n_bins=bins.n_bins, dk=bins.dk) as plan:
        host = plan.estimate_host((gal.x, gal.y, gal.z, gal.w, gal.nbar), (ran.x, ran.y, ran.z, ran.w, ran.nbar))
        again = plan.estimate_host((gal.x, gal.y, gal.z, gal.w, gal.nbar), (ran.x, ran.y, ran.z, ran.w, ran.nbar))
    compare(host, ref, 4, "host_entry")
    compare(again, ref, 4, "host_entry_repeat")


def test_particle_on_node_from_above_is_inside():
    """Particles on (within float rounding of) interior node positions of a box whose
    node positions are not exact in binary deposit normally, with no particle
    reported outside the box."""
    n = 32
    lo = np.array([8.115091545104981, 7.96615813446045, 8.116680366516114])
    L = 1912.451478515625
    rng = np.random.default_rng(5)
    mk = lambda k: synth.Catalog.from_positions(lo + rng.integers(1, n - 1, size=(k, 3)) * (L / n), 1.0, 1e-4)
    gal, ran = mk(2000), mk(10000)
    geo = synth.Geometry(tuple(lo), L, (0.0, 0.0, 0.0))
    bins = BinSpec(0.0, 0.005, 10)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="tsc", interlace=True)
    res = run_gpu(gal, ran, geo, n, bins, "tsc", True)
    assert res.status == 0
    compare(res, ref, 4, "near_nodes")


@pytest.mark.parametrize("kind,interlace,compensate", [("cic", True, False), ("tsc", False, True),
                                                       ("ngp", False, True)])
def test_offset_shells_and_window_options(kind, interlace, compensate):
    """Shells starting above k = 0 with a width that does not divide the fundamental
    frequency, the last shell ending just below Nyquist, and the window compensation
    switched on or off; 64^3 in an off-centre box (a ragged tail of pencil blocks)."""
    gal, ran, geo = synth.poisson_cube(15_000, 60_000, side=700.0, center=(900.0, -300.0, 450.0), seed=91)
    n = 64
    k_nyq = np.pi * n / geo.box_len
    k_min, dk = 0.013, 0.0123
    nb = int(np.floor((k_nyq - k_min) / dk))
    bins = BinSpec(k_min, dk, nb)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, interlace=interlace, compensate=compensate)
    res = run_gpu(gal, ran, geo, n, bins, kind, interlace, compensate=compensate)
    compare(res, ref, 4, f"offset_shells_{kind}_{interlace}_{compensate}")


@pytest.mark.parametrize("seed", [92, 93, 94, 95])
def test_many_shells_at_the_limit(seed):
    """4096 shells (the ABI's limit), most of them empty at this mesh: every shell
    holds one |k| value and a few dozen modes, so P_4 rests on a handful of terms
    of either sign -- the case that shows float shell sums (their error alone
    reached 1e-4 here in a float32 emulation; the compensated sums remove it)."""
    gal, ran, geo = synth.poisson_cube(5_000, 25_000, seed=seed)
    n = 32
    bins = BinSpec(0.0, np.pi * n / geo.box_len / 4096, 4096)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="cic")
    res = run_gpu(gal, ran, geo, n, bins, "cic")
    assert res.k.size == 4096
    compare(res, ref, 4, f"4096_shells_seed{seed}")


def test_shell_limit_at_the_largest_mesh():
    """The x stage keeps every shell's compensated sums in shared memory: 4096 shells
    (the ABI's limit) fit even at 1024^3, and one more is refused on the host."""
    with ys.Plan(1024, (0.0, 0.0, 0.0), 1000.0, assign="cic", dk=1e-4, n_bins=4096) as plan:
        assert plan.n_bins == 4096
    with pytest.raises(ys.YstatError) as ei:
        ys.Plan(1024, (0.0, 0.0, 0.0), 1000.0, assign="cic", dk=1e-4, n_bins=4097)
    assert ei.value.status == ys.ystat.YS_ERR_ARG


@pytest.mark.parametrize("n,kind,interlace", [(64, "tsc", True), (128, "cic", False), (96, "ngp", True)])
def test_direct_assignment_matches_oracle_and_sorted(n, kind, interlace):
    """The direct assignment (global reductions into an L2-resident mesh) against the
    oracle, and against the tile-sorted assignment (two float evaluations: twice the
    bar); particles outside the box are still reported."""
    gal, ran, geo = synth.zeldovich_cube(60_000, 300_000, seed=77)
    bins = BinSpec.up_to(np.pi * n / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, interlace=interlace)
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign=kind, interlace=interlace, dk=bins.dk,
                 n_bins=bins.n_bins, stream=torch.cuda.current_stream().cuda_stream) as plan:
        dg, dr = to_dev(gal), to_dev(ran)
        plan.assign(dg, dr)
        sorted_res = plan.measure()
        plan.set_direct_assign(True)
        plan.assign(dg, dr)
        direct_res = plan.measure()
    compare(direct_res, ref, 4, f"direct_{n}_{kind}_{interlace}")
    has = ref.n_modes > 0
    raw = np.where(has, ref.sum0 / np.where(has, ref.n_modes, 1) / ref.norm.I, 0.0)
    for l in (0, 2, 4):
        a, b = getattr(sorted_res, f"p{l}"), getattr(direct_res, f"p{l}")
        sel = has & (np.abs(a) > 1e-2 * raw)
        assert np.max(np.abs(a[sel] - b[sel]) / np.abs(a[sel])) <= 2 * TOL
    out = synth.poisson_cube(100, 500, seed=2)
    g2, r2, geo2 = out
    g2.x[0] = geo2.box_min[0] - 5.0
    with ys.Plan(32, geo2.box_min, geo2.box_len, geo2.observer, dk=0.05, n_bins=4,
                 stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.set_direct_assign(True)
        plan.assign(to_dev(g2), to_dev(r2))
        with pytest.raises(ys.YstatError) as ei:
            plan.measure()
        assert ei.value.status == ys.ystat.YS_ERR_ARG


def test_direct_assignment_refused_for_large_meshes():
    with ys.Plan(512, (0.0, 0.0, 0.0), 1000.0, dk=0.1, n_bins=4) as plan:
        with pytest.raises(ys.YstatError) as ei:
            plan.set_direct_assign(True)
        assert ei.value.status == ys.ystat.YS_ERR_UNSUPPORTED
