"""Seeded synthetic workloads: the paper-shaped stand-in (Sec. 4's single survey mock
of ~525 000 galaxies, ten times as many randoms, a 3500 Mpc/h box) has the stated
sizes, geometry and weights."""
import math

import numpy as np

import synth


def test_paper_shaped_cap():
    gal, ran, geo, st = synth.workload("paper512_cic")
    assert (gal.n, ran.n) == (525_000, 5_250_000)
    assert geo.box_len == 3500.0 and geo.observer == (0.0, 0.0, 0.0)
    assert st["n_mesh"] == 512 and st["assign"] == "cic" and not st["interlace"]
    lo = np.asarray(geo.box_min)
    cos_half = 1.0 - 7000.0 * (math.pi / 180.0) ** 2 / (2.0 * math.pi)   # a 7000 deg^2 cap
    for cat in (gal, ran):
        p = cat.positions().astype(np.float64)
        assert np.all(p >= lo) and np.all(p < lo + geo.box_len)
        r = np.linalg.norm(p, axis=1)
        assert r.min() >= 1100.0 - 1e-3 and r.max() < 1900.0 + 1e-3
        assert np.all(p[:, 2] / r >= cos_half - 1e-6)                   # inside the cap about +z
        np.testing.assert_allclose(cat.w, 1.0 / (1.0 + cat.nbar.astype(np.float64) * 2.0e4), rtol=1e-6)
    # galaxies and randoms follow the same radial selection, so their mean nbar agree
    assert abs(np.mean(ran.nbar) / np.mean(gal.nbar) - 1.0) < 0.05
