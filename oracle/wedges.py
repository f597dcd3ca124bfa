"""Power-spectrum wedges (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 5 of the paper replaces the Legendre weight of the estimator (Eq. 4) by top hats
in mu, 0 <= mu <= 1/2 (P_perp) and 1/2 < mu <= 1 (P_para), Eqs. 14-15, and
approximates both by the first three even multipoles, Eqs. 16-17 (the coefficients
are the averages of L_2 and L_4 over each half of the mu range).

``wedges_from_multipoles``: Eqs. 16-17.
``wedges_sum_gal``: Eqs. 14-15 themselves, as a direct sum over galaxies and randoms.
In the Yamamoto form the top hat, like L_l in Eq. 4, sits on one particle of each
pair, with mu = k_hat . r_hat of that particle (mu = 0 at r = 0):
    B_perp(k) = sum_p s_p w_p Theta(|k_hat . r_hat_p| <= 1/2) e^{-i k.(x_p - box_min)},
    P_perp = (2 / I) <Re A_0 B_perp^*> - S / I,
and B_para, P_para alike with Theta(1/2 < |k_hat . r_hat_p| <= 1).  The factor
2 = 1 / int dmu over each half normalises the top hat as (2l + 1) does L_l, and S / I
is the monopole's shot noise (Eqs. 14-15 subtract P_0^noise from both).  The two top
hats add up to 1, so B_perp + B_para = A_0 and P_perp + P_para = 2 P_0; both sums are
formed separately, so that identity checks them.

Pinned by: the coefficients of Eqs. 16-17 against numerical averages of the Legendre
polynomials over the two ranges; the exact wedges of a P(k, mu) that is a polynomial
of degree 4 in mu (for which the truncation at l = 4 is exact); for the direct sum,
P_perp + P_para = 2 P_0 of the galaxy sum (``direct.sum_gal``), and one particle of
unit weight, for which Re A_0 B_perp^* is the top hat itself and the shell average is
a count of lattice directions (tests/test_oracle_wedges.py).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .binning import BinSpec, bin_sums, kfund
from .direct import _valid_modes
from .normalization import Norm, catalog_sums


def wedges_from_multipoles(p0, p2, p4):
    """(P_perp, P_para) of Eqs. 16-17."""
    p0, p2, p4 = (np.asarray(a, dtype=np.float64) for a in (p0, p2, p4))
    return p0 - 3.0 / 8.0 * p2 + 15.0 / 128.0 * p4, p0 + 3.0 / 8.0 * p2 - 15.0 / 128.0 * p4


@dataclasses.dataclass
class Wedges:
    k: np.ndarray
    n_modes: np.ndarray
    p_perp: np.ndarray
    p_para: np.ndarray
    sum_a0: np.ndarray     # sum_w |A_0|^2 per shell
    sum_perp: np.ndarray   # sum_w Re A_0 B_perp^* per shell
    sum_para: np.ndarray   # sum_w Re A_0 B_para^* per shell
    norm: Norm


def wedges_sum_gal(gal, ran, geo, n_mesh: int, bins: BinSpec, alpha=None, mu_edge: float = 0.5,
                   chunk: int = 512) -> Wedges:
    """Eqs. 14-15 by direct summation over the half-grid modes of an n_mesh^3 FFT."""
    norm = catalog_sums(gal, ran, alpha)
    M, bidx, w, kmag, _ = _valid_modes(n_mesh, geo.box_len, bins)
    kvec = M * kfund(geo.box_len)
    khat = kvec / np.linalg.norm(kvec, axis=1)[:, None]
    lo = np.asarray(geo.box_min, dtype=np.float64)
    obs = np.asarray(geo.observer, dtype=np.float64)
    pos = np.concatenate([gal.positions(), ran.positions()]).astype(np.float64)
    wts = np.concatenate([gal.w.astype(np.float64), -norm.alpha * ran.w.astype(np.float64)])
    A0 = np.zeros(M.shape[0], dtype=np.complex128)
    Bp = np.zeros(M.shape[0], dtype=np.complex128)
    Bq = np.zeros(M.shape[0], dtype=np.complex128)
    for s in range(0, pos.shape[0], chunk):
        p = pos[s:s + chunk] - lo
        r = pos[s:s + chunk] - obs
        rn = np.linalg.norm(r, axis=1)
        rhat = np.where(rn[:, None] > 0, r / np.where(rn > 0, rn, 1.0)[:, None], 0.0)
        term = np.exp(-1j * (p @ kvec.T)) * wts[s:s + chunk, None]
        mu = rhat @ khat.T
        A0 += term.sum(axis=0)
        Bp += np.where(np.abs(mu) <= mu_edge, term, 0.0).sum(axis=0)
        Bq += np.where(np.abs(mu) > mu_edge, term, 0.0).sum(axis=0)
    nb = bins.n_bins
    nmodes = bin_sums(np.ones_like(kmag), bidx, w, nb)
    ksum = bin_sums(kmag, bidx, w, nb)
    s0 = bin_sums((A0 * np.conj(A0)).real, bidx, w, nb)
    sp = bin_sums((A0 * np.conj(Bp)).real, bidx, w, nb)
    sq = bin_sums((A0 * np.conj(Bq)).real, bidx, w, nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        p_perp = (1.0 / mu_edge) / norm.I * sp / nmodes - norm.S / norm.I
        p_para = (1.0 / (1.0 - mu_edge)) / norm.I * sq / nmodes - norm.S / norm.I
        kmean = ksum / nmodes
    return Wedges(kmean, nmodes, p_perp, p_para, s0, sp, sq, norm)
