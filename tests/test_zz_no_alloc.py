"""ys_assign_noalloc: the assignment step for callers that must not allocate device
memory after set-up (its sorting scratch lives in one static 64 MiB device array
instead of plan-owned cudaMalloc buffers).

Checked through the C ABI against ys_assign on the same catalogue: after each of two
calls in a row, ys_measure_multipoles must give the same multipoles within the parity
bar used everywhere else (1e-4 relative where |P_l| > 1e-2 of the raw monopole).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
ys = pytest.importorskip("paper_1505_05341_gb300")
from paper_1505_05341_gb300 import ystat  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev(c):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (c.x, c.y, c.z, c.w, c.nbar)]


def _cat(ts):
    c = ystat.YsCatalog()
    c.x, c.y, c.z, c.w, c.nbar = [t.data_ptr() for t in ts]
    c.n = int(ts[0].shape[0])
    return c


def _plan(geo, max_particles):
    return ys.Plan(64, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, ell_max=4,
                   dk=0.01, n_bins=14, max_particles=max_particles,
                   stream=torch.cuda.current_stream().cuda_stream)


def _same(a, b):
    np.testing.assert_array_equal(a.n_modes, b.n_modes)
    has = a.n_modes > 0
    raw = a.p0 + a.shot_noise          # monopole before the shot noise is subtracted
    for l in (0, 2, 4):
        x, y = getattr(a, f"p{l}"), getattr(b, f"p{l}")
        sel = has & (np.abs(x) > 1e-2 * np.abs(raw))
        assert sel.any()
        assert np.max(np.abs(y[sel] - x[sel]) / np.abs(x[sel])) <= TOL, l
    assert b.alpha == pytest.approx(a.alpha, rel=1e-12)
    assert b.norm_I == pytest.approx(a.norm_I, rel=1e-12)


def test_noalloc_matches_assign_twice_in_a_row():
    lib = ys.load_library()
    cats = [synth.poisson_cube(20_000, 100_000, side=1000.0, center=(0.0, 0.0, 0.0), seed=s)
            for s in (71, 72)]
    geo = cats[0][2]
    with _plan(geo, 0) as fresh, _plan(geo, 200_000) as ref:
        for gal, ran, _ in cats:
            dg, dr = _dev(gal), _dev(ran)
            cg, cr = _cat(dg), _cat(dr)
            assert lib.ys_assign(ref._h, ctypes.byref(cg), ctypes.byref(cr)) == ystat.YS_OK
            want = ref.measure()
            st = lib.ys_assign_noalloc(fresh._h, ctypes.byref(cg), ctypes.byref(cr))
            assert st == ystat.YS_OK, lib.ys_last_cuda_error()
            got = fresh.measure()
            _same(want, got)


def test_noalloc_rejects_oversized_catalogue():
    lib = ys.load_library()
    gal, ran, geo = synth.poisson_cube(100_000, 500_000, side=1000.0, center=(0.0, 0.0, 0.0), seed=73)
    with _plan(geo, 0) as plan:
        dg, dr = _dev(gal), _dev(ran)
        st = lib.ys_assign_noalloc(plan._h, ctypes.byref(_cat(dg)), ctypes.byref(_cat(dr)))
        assert st == ystat.YS_ERR_UNSUPPORTED
        assert b"limit" in lib.ys_last_cuda_error()
        with pytest.raises(ys.YstatError):
            plan.measure()  # nothing was assigned
