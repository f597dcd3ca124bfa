"""The failure path of the y,z stage's bounded waits, exercised without any fault.

ys_plan_set_fault_injection shortens the bound of every wait in the persistent
y,z kernel to 20 ms and makes the row items of one x-plane withhold their
completion signal: the column items of that plane then wait for a counter that
nothing raises, give up at the bound, set the error flag, and every other CTA
leaves at its next wait.  The call must report YS_ERR_TIMEOUT within about a
second, and the same plan, with the hook switched off, must measure correctly
again.  No copy, barrier or memory access is withheld or broken: only the
release of one completion counter is skipped.  This file is collected just
before the no-allocation test, so a failure here stops a -x run late."""
import time

import numpy as np
import pytest

import oracle
import synth
from oracle.binning import BinSpec

torch = pytest.importorskip("torch")
ys = pytest.importorskip("paper_1505_05341_gb300")

pytestmark = pytest.mark.gpu


def _dev(c):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (c.x, c.y, c.z, c.w, c.nbar))


@pytest.mark.parametrize("skip_plane", [5, 64 + 3])
def test_withheld_completion_times_out_then_recovers(skip_plane):
    gal, ran, geo = synth.poisson_cube(20_000, 100_000, side=800.0, center=(500.0, 0.0, 0.0), seed=31)
    n = 64
    bins = BinSpec.up_to(np.pi * n / geo.box_len, 0.01)
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, ell_max=4,
                 dk=bins.dk, n_bins=bins.n_bins, stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.assign(_dev(gal), _dev(ran))
        good = plan.measure()                       # captured graph, no hook
        plan.set_fault_injection(20_000_000, skip_plane)   # 20 ms bound
        t0 = time.perf_counter()
        with pytest.raises(ys.YstatError) as ei:
            plan.measure()
        elapsed = time.perf_counter() - t0
        assert ei.value.status == ys.ystat.YS_ERR_TIMEOUT
        assert elapsed < 5.0, elapsed
        plan.set_fault_injection(0, -1)             # back to the default 1 s bound
        again = plan.measure()
        np.testing.assert_array_equal(again.n_modes, good.n_modes)
        np.testing.assert_allclose(again.p0, good.p0, rtol=1e-5, equal_nan=True)
        np.testing.assert_allclose(again.p4, good.p4, rtol=1e-4, atol=1e-6 * np.nanmax(np.abs(good.p0)),
                                   equal_nan=True)
    # the recovered measurement meets the parity bar against the oracle (shells where
    # |P_l| > 1e-2 of the raw monopole, as in every parity test)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="tsc", interlace=True)
    has = ref.n_modes > 0
    raw = np.where(has, ref.sum0 / np.where(has, ref.n_modes, 1) / ref.norm.I, 0.0)
    for l in (0, 2, 4):
        g, o = getattr(again, f"p{l}"), getattr(ref, f"p{l}")
        sel = has & (np.abs(o) > 1e-2 * raw)
        assert np.max(np.abs(g[sel] - o[sel]) / np.abs(o[sel])) <= 1e-4, l


def test_out_of_range_hook_values_rejected():
    with ys.Plan(32, (0.0, 0.0, 0.0), 100.0, assign="cic", dk=0.05, n_bins=4) as plan:
        for limit, plane in ((0, 32), (0, -2), (20_000_000_000, -1)):
            with pytest.raises(ys.YstatError) as ei:
                plan.set_fault_injection(limit, plane)
            assert ei.value.status == ys.ystat.YS_ERR_ARG
