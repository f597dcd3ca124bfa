"""Direct-sum routes to the Yamamoto multipoles (oracle; FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 4 compares the FFT-based method with two plain sums over the same k modes:
* sum-gal: A_n(k) = sum_i s_i w_i (k_hat . r_hat_i)^n e^{-i k.x_i} over galaxies
  (s = +1) and randoms (s = -alpha), r_i = x_i - observer  (Eq. 5 with F of Eq. 1);
* sum-grid: the same sum over mesh nodes carrying F, r = node - observer.
(k_hat . r_hat)^n is evaluated directly per (mode, point); it is 0 at r = 0 for
n > 0.  Both use the half-grid modes and shell binning of ``binning``, and the
Legendre combination of Eqs. (6)-(8).

With ``legendre=True`` sum-gal instead forms A_l^L(k) = sum s w L_l(k_hat.r_hat)
e^{-ik.x} with scipy's Legendre polynomials and P_l = (2l+1)/I <Re A_0 A_l^L*>
(P_0 minus S/I): Eq. (4) as written, which pins the coefficients of Eqs. (6)-(8).

Cost is O(points x modes); use for small cases (<= 32^3 modes, ~1e4 points).
"""
from __future__ import annotations

import numpy as np
import scipy.special

from .binning import BinSpec, bin_sums, half_modes, kfund, mode_bins
from .estimator import Multipoles, legendre_combination, node_offsets, p6_combination, window
from .normalization import catalog_sums


def _valid_modes(n, box_len, bins):
    bidx, w, kmag = mode_bins(n, box_len, bins)
    mx, my, mz, _ = half_modes(n)
    sel = bidx >= 0
    M = np.stack([np.broadcast_to(mx, bidx.shape)[sel], np.broadcast_to(my, bidx.shape)[sel],
                  np.broadcast_to(mz, bidx.shape)[sel]], axis=1).astype(np.float64)
    return M, bidx[sel], w[sel], kmag[sel], sel


def _point_sums(pos, wts, rel, kvec, ell_max, legendre, chunk=512):
    """sum_p wts_p f(k_hat.r_hat_p) e^{-i k.pos_p} for f = mu^0, mu^2, mu^4, mu^6 (up to
    ell_max; or the Legendre polynomials), for every k in kvec (M, 3)."""
    M = kvec.shape[0]
    kn = np.linalg.norm(kvec, axis=1)
    khat = kvec / kn[:, None]
    outs = {n: np.zeros(M, dtype=np.complex128) for n in (0, 2, 4, 6) if n <= ell_max}
    for s in range(0, pos.shape[0], chunk):
        p = pos[s:s + chunk]
        r = rel[s:s + chunk]
        ww = wts[s:s + chunk]
        rn = np.linalg.norm(r, axis=1)
        rhat = np.where(rn[:, None] > 0, r / np.where(rn > 0, rn, 1.0)[:, None], 0.0)
        ph = np.exp(-1j * (p @ kvec.T)) * ww[:, None]
        mu = rhat @ khat.T
        zero_r = (rn == 0)[:, None]
        for n in outs:
            if legendre:
                f = scipy.special.eval_legendre(n, mu)
                if n > 0:
                    f = np.where(zero_r, 0.0, f)
            else:
                f = mu ** n if n > 0 else np.ones_like(mu)
            outs[n] += np.sum(f * ph, axis=0)
    return outs


def _finish(A, bidx, w, kmag, bins, norm, legendre, ell_max):
    nb = bins.n_bins
    nmodes = bin_sums(np.ones_like(kmag), bidx, w, nb)
    ksum = bin_sums(kmag, bidx, w, nb)
    A0 = A[0]
    s0 = bin_sums((A0 * np.conj(A0)).real, bidx, w, nb)
    s2 = bin_sums((A0 * np.conj(A[2])).real, bidx, w, nb) if ell_max >= 2 else np.zeros(nb)
    s4 = bin_sums((A0 * np.conj(A[4])).real, bidx, w, nb) if ell_max >= 4 else np.zeros(nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = ksum / nmodes
        s6 = bin_sums((A0 * np.conj(A[6])).real, bidx, w, nb) if ell_max >= 6 else None
        p6 = None
        if legendre:
            p0 = (s0 / nmodes - norm.S) / norm.I
            p2 = 5.0 / norm.I * s2 / nmodes
            p4 = 9.0 / norm.I * s4 / nmodes
            if s6 is not None:
                p6 = 13.0 / norm.I * s6 / nmodes
        else:
            p0, p2, p4 = legendre_combination(s0, s2, s4, nmodes, norm)
            if s6 is not None:
                p6 = p6_combination(s0, s2, s4, s6, nmodes, norm)
    return Multipoles(kmean, nmodes, p0, p2, p4, s0, s2, s4, norm, modes=A, p6=p6, sum6=s6)


def sum_gal(gal, ran, geo, n_mesh: int, bins: BinSpec, alpha=None, ell_max: int = 4,
            legendre: bool = False) -> Multipoles:
    """sum-gal over the half-grid modes of an n_mesh^3 FFT (no mesh, no window)."""
    norm = catalog_sums(gal, ran, alpha)
    M, bidx, w, kmag, _ = _valid_modes(n_mesh, geo.box_len, bins)
    kvec = M * kfund(geo.box_len)
    lo = np.asarray(geo.box_min, dtype=np.float64)
    obs = np.asarray(geo.observer, dtype=np.float64)
    pos = np.concatenate([gal.positions(), ran.positions()]).astype(np.float64)
    wts = np.concatenate([gal.w.astype(np.float64), -norm.alpha * ran.w.astype(np.float64)])
    A = _point_sums(pos - lo, wts, pos - obs, kvec, ell_max, legendre)
    return _finish(A, bidx, w, kmag, bins, norm, legendre, ell_max)


def sum_grid(meshes, gal, ran, geo, n_mesh: int, bins: BinSpec, assign: str = "cic",
             compensate: bool = True, alpha=None, ell_max: int = 4) -> Multipoles:
    """sum-grid: direct sum over the filled nodes of the given mesh(es).  A second
    mesh is taken as the interlaced one, with its nodes at +H/2."""
    norm = catalog_sums(gal, ran, alpha)
    n = n_mesh
    L = geo.box_len
    H = L / n
    M, bidx, w, kmag, sel = _valid_modes(n, L, bins)
    kvec = M * kfund(L)
    acc = None
    for j, F in enumerate(meshes):
        il = j == 1
        ox, oy, oz = node_offsets(geo.box_min, L, n, geo.observer, il)
        ix, iy, iz = np.nonzero(F)
        vals = F[ix, iy, iz]
        s = 0.5 if il else 0.0
        pos = np.stack([(ix + s) * H, (iy + s) * H, (iz + s) * H], axis=1)
        rel = np.stack([ox[ix], oy[iy], oz[iz]], axis=1)
        A = _point_sums(pos, vals, rel, kvec, ell_max, legendre=False)
        acc = A if acc is None else {k: acc[k] + A[k] for k in acc}
    if len(meshes) == 2:
        acc = {k: 0.5 * v for k, v in acc.items()}
    if compensate:
        Wk = window(n, assign)[sel]
        acc = {k: v / Wk for k, v in acc.items()}
    return _finish(acc, bidx, w, kmag, bins, norm, False, ell_max)
