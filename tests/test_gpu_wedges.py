"""Wedges (Eqs. 16-17) from the GPU's result rows, against the oracle's combination:
on synthetic rows exactly (up to FP64 rounding), and on a measurement of a clustered
mock against the oracle's own multipoles at the parity bar."""
import numpy as np
import pytest

import oracle
import synth
from oracle.binning import BinSpec
from oracle.wedges import wedges_from_multipoles
from test_gpu_parity import TOL

torch = pytest.importorskip("torch")
ys = pytest.importorskip("paper_1505_05341_gb300")

pytestmark = pytest.mark.gpu


def test_wedges_of_result_rows():
    rng = np.random.default_rng(5)
    n_cat, nb = 3, 29
    stride = 5 * nb + 9   # rows spaced wider than they need
    rows = rng.standard_normal((n_cat, stride)) * 1e4
    rows[1, 2 * nb + 4] = np.nan
    d_rows = torch.from_numpy(rows).cuda()
    out = torch.empty((n_cat, 2, nb), dtype=torch.float64, device="cuda")
    ys.wedges(d_rows, nb, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for c in range(n_cat):
        perp, para = wedges_from_multipoles(rows[c, 2 * nb:3 * nb], rows[c, 3 * nb:4 * nb], rows[c, 4 * nb:5 * nb])
        for g, w in ((got[c, 0], perp), (got[c, 1], para)):
            assert np.array_equal(np.isnan(g), np.isnan(w))
            ok = ~np.isnan(w)
            scale = np.nanmax(np.abs(rows[c, 2 * nb:5 * nb]))
            assert np.abs(g[ok] - w[ok]).max() <= 1e-14 * scale


def test_wedges_of_a_clustered_mock_match_oracle():
    gal, ran, geo = synth.zeldovich_cube(150_000, 750_000, seed=21)
    n = 64
    bins = BinSpec.up_to(np.pi * n / geo.box_len, 0.01)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="tsc", interlace=True)
    with ys.Plan(n, geo.box_min, geo.box_len, geo.observer, assign="tsc", interlace=True, dk=bins.dk,
                 n_bins=bins.n_bins, stream=torch.cuda.current_stream().cuda_stream) as plan:
        plan.assign(*[tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                            for a in (c.x, c.y, c.z, c.w, c.nbar)) for c in (gal, ran)])
        row = torch.empty((1, 5 * bins.n_bins + 5), dtype=torch.float64, device="cuda")
        plan.measure_async(row[0])
        out = torch.empty((1, 2, bins.n_bins), dtype=torch.float64, device="cuda")
        ys.wedges(row, bins.n_bins, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy()[0]
    perp, para = wedges_from_multipoles(ref.p0, ref.p2, ref.p4)
    has = ref.n_modes > 0
    raw = np.where(has, ref.sum0 / np.where(has, ref.n_modes, 1) / ref.norm.I, 0.0)
    for g, w, name in ((got[0], perp, "perp"), (got[1], para, "para")):
        sel = has & (np.abs(w) > 1e-2 * raw)
        assert sel.sum() > 3, name
        rel = np.abs(g[sel] - w[sel]) / np.abs(w[sel])
        print(name, "worst rel err", rel.max())
        assert rel.max() <= TOL, name
