"""The library's k_x-power grouping (csrc/gen_group_table.py: 16 basis fields for
l <= 4, 29 for l <= 6) reproduces the oracle's literal 22-field A_2 and A_4 of
Eqs. (10) and (12), and its 28-field A_6, at every mode, including an observer
sitting exactly on a mesh node (host-side check)."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.estimator import mesh_transforms, node_offsets

HERE = os.path.dirname(os.path.abspath(__file__))
GEN = os.path.join(HERE, "..", "paper_1505_05341_gb300", "csrc", "gen_group_table.py")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_group_table", GEN)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("center", [(0.0, 0.0, 0.0), (300.0, -120.0, 45.0)])
def test_grouping_reproduces_eqs_10_12(center):
    G = _gen()
    n = 16
    gal, ran, geo = synth.poisson_cube(500, 2500, side=160.0, center=center, seed=3)
    nm = oracle.catalog_sums(gal, ran)
    F = oracle.assign_mesh(gal, ran, nm.alpha, geo.box_min, geo.box_len, n, "cic")
    rx, ry, rz = node_offsets(geo.box_min, geo.box_len, n, geo.observer, False)
    if center == (0.0, 0.0, 0.0):
        assert np.any(rx == 0) and np.any(ry == 0) and np.any(rz == 0)
    T = mesh_transforms(F, rx, ry, rz, 6, 1)
    X, Y, Z = rx[:, None, None], ry[None, :, None], rz[None, None, :]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    inv = np.where(r > 0, 1 / np.where(r > 0, r, 1), 0)
    xh, yh, zh = X * inv, Y * inv, Z * inv
    m = np.fft.fftfreq(n, 1 / n)
    kx, ky, kz = m[:, None, None], m[None, :, None], np.arange(n // 2 + 1)[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    for ell in (2, 4, 6):
        bs, tab, gs = G.basis(ell), G.table(ell), G.groups(ell)
        assert len(bs) == {2: 7, 4: 16, 6: 29}[ell]
        psi = []
        for (a, b, c, d) in bs:
            f = F if d == 0 else (np.where(r > 0, F, 0.0) if d == -1 else F * xh ** a * yh ** b * zh ** c)
            psi.append(np.fft.fftn(f, axes=(1, 2))[:, :, :n // 2 + 1])
        grp = [np.zeros_like(psi[0]) for _ in gs]
        for (gi, beta), poly in tab.items():
            grp[gi] = grp[gi] + sum(float(v) * ky ** b * kz ** c for (b, c), v in poly.items()) * psi[beta]
        grpx = [np.fft.fft(g_, axis=0) for g_ in grp]
        np.testing.assert_allclose(grpx[0], T["A0"], rtol=0, atol=1e-12 * np.abs(T["A0"]).max())
        for nn, key in ((2, "A2"), (4, "A4"), (6, "A6")):
            if nn > ell:
                continue
            acc = sum(kx ** p * grpx[gs.index((nn, p))] for p in range(nn + 1))
            ref = T[key] * k2 ** (nn // 2)
            assert np.max(np.abs(acc - ref)) <= 1e-12 * np.max(np.abs(ref))
