"""Shared randoms (Sec. 4: catalogues that share one random catalogue need it only
once): ys_randoms_cache + ys_assign_cached against the FP64 oracle and against
ys_assign on the same inputs, through the C ABI."""
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


def _check(res, ref, label, tol=TOL):
    np.testing.assert_array_equal(res.n_modes, ref.n_modes)
    has = ref.n_modes > 0
    raw = np.where(has, ref.sum0 / np.where(has, ref.n_modes, 1) / ref.norm.I, 0.0)
    assert res.alpha == pytest.approx(ref.norm.alpha, rel=1e-12)
    assert res.norm_I == pytest.approx(ref.norm.I, rel=1e-12)
    worst = {}
    for l in (0, 2, 4):
        g, o = getattr(res, f"p{l}"), getattr(ref, f"p{l}")
        sel = has & (np.abs(o) > 1e-2 * raw)
        rel = np.abs(g[sel] - o[sel]) / np.abs(o[sel])
        worst[l] = float(rel.max())
        assert rel.max() <= tol, (label, l, rel.max())
    print(f"{label}: worst rel err per multipole {worst}")


@pytest.mark.parametrize("n,kind,interlace,alpha", [(64, "tsc", True, -1.0), (96, "cic", False, 0.21)])
def test_two_catalogues_against_one_random_catalogue(n, kind, interlace, alpha):
    """Two clustered galaxy catalogues measured against the same kept randoms: each
    equals the oracle, and ys_assign with the randoms passed again (two float
    evaluations: twice the bar)."""
    g1, ran, geo = synth.zeldovich_cube(40_000, 200_000, seed=81)
    g2, _, _ = synth.zeldovich_cube(30_000, 10, seed=82)
    bins = BinSpec.up_to(np.pi * n / geo.box_len, 0.01)
    a = None if alpha < 0 else alpha
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign=kind, interlace=interlace, ell_max=4,
                 dk=bins.dk, n_bins=bins.n_bins, alpha=alpha,
                 stream=torch.cuda.current_stream().cuda_stream) as plan:
        dran = to_dev(ran)
        plan.cache_randoms(dran)
        for k, gal in enumerate((g1, g2)):
            dgal = to_dev(gal)
            plan.assign_cached(dgal)
            cached = plan.measure()
            plan.assign(dgal, dran)
            plain = plan.measure()
            ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign=kind, interlace=interlace, alpha=a)
            _check(cached, ref, f"cached_{n}_{k}")
            _check(plain, ref, f"plain_{n}_{k}")
            has = ref.n_modes > 0
            raw = plain.p0 + plain.shot_noise
            for l in (0, 2, 4):
                x, y = getattr(plain, f"p{l}"), getattr(cached, f"p{l}")
                sel = has & (np.abs(x) > 1e-2 * np.abs(raw))
                assert np.max(np.abs(x[sel] - y[sel]) / np.abs(x[sel])) <= 2 * TOL


def test_cached_assign_needs_a_cache():
    gal, ran, geo = synth.poisson_cube(100, 500, seed=83)
    with ys.Plan(32, geo.box_min, geo.box_len, geo.observer, assign="cic", dk=0.02, n_bins=5,
                 stream=torch.cuda.current_stream().cuda_stream) as plan:
        with pytest.raises(ys.YstatError) as ei:
            plan.assign_cached(to_dev(gal))
        assert ei.value.status == ys.ystat.YS_ERR_STATE
        plan.cache_randoms(to_dev(ran))
        with pytest.raises(ys.YstatError) as ei:   # the cache used the plan's sums
            plan.measure()
        assert ei.value.status == ys.ystat.YS_ERR_STATE
