"""FFT-based Yamamoto multipoles, written out literally (oracle; FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Steps, in the paper's order:
1. F on the mesh (Eq. 1 with cell sums; ``assignment.assign_mesh``), alpha, I, S
   (``normalization.catalog_sums``).
2. The LOS-weighted fields at the mesh nodes, r = node - observer (weight 0 at
   r = 0): F (for A_0), F r_i r_j / r^2 (the six B_ij of Eq. 11) and
   F r_i^2 r_j r_l / r^4 (the fifteen C_ijl of Eq. 13) -- all 22, no regrouping.
3. One FP64 real-to-complex FFT per field (scipy.fft.rfftn, sign e^{-ik.x}).
   A_n(k) of Eq. (5) carries e^{+ik.r}; the estimator only uses Re(A_0 A_l^*), which
   is the same at k and -k for even n, so the FFT sign does not matter.
4. A_2 from Eq. (10) and A_4 from Eq. (12), term by term (``terms``).  With
   ell_max = 6 also A_6 from the 28 fields F r_x^a r_y^b r_z^c / r^6 (the same
   decomposition one order up, ``terms.A6_TERMS``) and P_6 (``p6_combination``).
5. Interlacing (a reading; the paper uses one CIC mesh): the second mesh has nodes
   at +H/2, so its transform carries the phase e^{-i k.(H/2)(1,1,1)};
   A = (A^(1) + e^{-i k.(H/2)(1,1,1)} A^(2)) / 2.
6. Window compensation (Sec. 4 cites Jing 2005 without a formula; reading):
   A_n /= prod_i [sin(k_i H/2)/(k_i H/2)]^p with p = 1, 2, 3 for NGP, CIC, TSC.
7. Eqs. (6)-(8) with Re(.), the shell mean over the half-grid modes (``binning``),
   a single 1/I normalisation (F is used without its I^{-1/2}), and the shot noise
   S/I subtracted from P_0 only (Eq. 3; negligible for l > 0 per Sec. 2):
     P_0 = <|A_0|^2>/I - S/I
     P_2 = 5/(2I) <Re A_0 (3 A_2 - A_0)^*>
     P_4 = 9/(8I) <Re A_0 (35 A_4 - 30 A_2 + 3 A_0)^*>

Pinned by: equality with the direct sums of ``direct`` (NGP on nodes, and sum-grid
at every mode), the distant-observer closed form, observer invariance of P_0,
translation / axis-permutation invariance, the Poisson shot-noise closed form, and,
for interlacing and compensation, the exact alias sum of one particle (Poisson
summation of the kernel's analytic transform: the interlaced mean keeps the aliases
of even q_x + q_y + q_z, compensation divides by the q = 0 factor)
(tests/test_oracle_pins.py).
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np
import scipy.fft

from .assignment import ORDER, assign_mesh
from .binning import BinSpec, bin_sums, half_modes, mode_bins
from .normalization import Norm, catalog_sums
from .terms import A2_TERMS, A4_TERMS, A6_TERMS, field_monomial


@dataclasses.dataclass
class Multipoles:
    k: np.ndarray          # mean |k| per bin
    n_modes: np.ndarray    # weighted mode count per bin (full-grid count)
    p0: np.ndarray
    p2: np.ndarray
    p4: np.ndarray
    sum0: np.ndarray       # sum_w |A0|^2
    sum2: np.ndarray       # sum_w Re A0 A2^*
    sum4: np.ndarray       # sum_w Re A0 A4^*
    norm: Norm
    modes: dict | None = None
    p6: np.ndarray | None = None     # l = 6 (ell_max = 6 only)
    sum6: np.ndarray | None = None   # sum_w Re A0 A6^*


def legendre_combination(sum0, sum2, sum4, nmodes, norm: Norm):
    """Eqs. (6)-(8) from the binned sums."""
    with np.errstate(invalid="ignore", divide="ignore"):
        m0 = sum0 / nmodes
        m2 = sum2 / nmodes
        m4 = sum4 / nmodes
        p0 = (m0 - norm.S) / norm.I
        p2 = 2.5 / norm.I * (3.0 * m2 - m0)
        p4 = 1.125 / norm.I * (35.0 * m4 - 30.0 * m2 + 3.0 * m0)
    return p0, p2, p4


def p6_combination(sum0, sum2, sum4, sum6, nmodes, norm: Norm):
    """P_6 = 13/I <Re A_0 [L_6 combination]^*> with L_6(mu) = (231 mu^6 - 315 mu^4
    + 105 mu^2 - 5) / 16, the l = 6 term of Eq. (4) written with the mu-power sums."""
    with np.errstate(invalid="ignore", divide="ignore"):
        m0, m2, m4, m6 = (v / nmodes for v in (sum0, sum2, sum4, sum6))
        return 13.0 / 16.0 / norm.I * (231.0 * m6 - 315.0 * m4 + 105.0 * m2 - 5.0 * m0)


def node_offsets(box_min, box_len, n, observer, interlaced):
    """Per-axis node coordinates relative to the observer (FP64, 1-D each)."""
    H = box_len / n
    s = 0.5 if interlaced else 0.0
    i = np.arange(n, dtype=np.float64)
    return [box_min[d] + (i + s) * H - observer[d] for d in range(3)]


def _workers():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def window(n, kind):
    """prod_i sinc(pi m_i / N)^p on the half grid."""
    mx, my, mz, _ = half_modes(n)
    p = ORDER[kind]

    def s(m):
        x = np.pi * m.astype(np.float64) / n
        return np.where(m == 0, 1.0, np.sin(x) / np.where(m == 0, 1.0, x)) ** p

    return s(mx) * s(my) * s(mz)


def mesh_transforms(F, rx, ry, rz, ell_max, workers):
    """A_0, A_2 and A_4 of one mesh (half grid), A_2 and A_4 literally from the 22
    single-field FFTs of Eqs. (10) and (12)."""
    n = F.shape[0]
    A0 = scipy.fft.rfftn(F, workers=workers)
    out = {"A0": A0}
    if ell_max < 2:
        return out
    mx, my, mz, _ = half_modes(n)
    kx = mx.astype(np.float64)
    ky = my.astype(np.float64)
    kz = mz.astype(np.float64)
    k2 = kx * kx + ky * ky + kz * kz
    inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    X = rx[:, None, None]
    Y = ry[None, :, None]
    Z = rz[None, None, :]
    r2 = X * X + Y * Y + Z * Z
    inv_r2 = np.where(r2 > 0, 1.0 / np.where(r2 > 0, r2, 1.0), 0.0)
    comps = (X, Y, Z)
    kc = (kx, ky, kz)

    def assemble(terms, inv_rpow, inv_kpow):
        acc = np.zeros_like(A0)
        for coef, kp, name in terms:
            (a, b, c), _deg = field_monomial(name)
            field = F * (comps[0] ** a) * (comps[1] ** b) * (comps[2] ** c) * inv_rpow
            T = scipy.fft.rfftn(field, workers=workers)
            acc += coef * (kc[0] ** kp[0]) * (kc[1] ** kp[1]) * (kc[2] ** kp[2]) * T
        return acc * inv_kpow

    out["A2"] = assemble(A2_TERMS, inv_r2, inv_k2)
    if ell_max >= 4:
        out["A4"] = assemble(A4_TERMS, inv_r2 * inv_r2, inv_k2 * inv_k2)
    if ell_max >= 6:
        out["A6"] = assemble(A6_TERMS, inv_r2 ** 3, inv_k2 ** 3)
    return out


def fft_multipoles(gal, ran, geo, n_mesh: int, bins: BinSpec, assign: str = "cic",
                   interlace: bool = False, compensate: bool = True, ell_max: int = 4,
                   alpha: float | None = None, workers: int | None = None,
                   return_modes: bool = False, meshes=None) -> Multipoles:
    """The FFT-based estimator, all 1 + 6 + 15 fields per mesh (see module header)."""
    workers = workers or _workers()
    norm = catalog_sums(gal, ran, alpha)
    n = n_mesh
    L = geo.box_len
    per_mesh = []
    for j, il in enumerate([False, True] if interlace else [False]):
        F = meshes[j] if meshes is not None else assign_mesh(
            gal, ran, norm.alpha, geo.box_min, L, n, assign, interlaced=il)
        rx, ry, rz = node_offsets(geo.box_min, L, n, geo.observer, il)
        per_mesh.append(mesh_transforms(F, rx, ry, rz, ell_max, workers))
        del F
    mx, my, mz, _ = half_modes(n)
    A = per_mesh[0]
    if interlace:
        phase = np.exp(-1j * np.pi * (mx + my + mz).astype(np.float64) / n)
        A = {key: 0.5 * (per_mesh[0][key] + phase * per_mesh[1][key]) for key in A}
    if compensate:
        Wk = window(n, assign)
        A = {key: v / Wk for key, v in A.items()}
    bidx, w, kmag = mode_bins(n, L, bins)
    nb = bins.n_bins
    nmodes = bin_sums(np.ones_like(kmag), bidx, w, nb)
    ksum = bin_sums(kmag, bidx, w, nb)
    A0 = A["A0"]
    s0 = bin_sums((A0 * np.conj(A0)).real, bidx, w, nb)
    s2 = bin_sums((A0 * np.conj(A["A2"])).real, bidx, w, nb) if ell_max >= 2 else np.zeros(nb)
    s4 = bin_sums((A0 * np.conj(A["A4"])).real, bidx, w, nb) if ell_max >= 4 else np.zeros(nb)
    p0, p2, p4 = legendre_combination(s0, s2, s4, nmodes, norm)
    s6 = p6 = None
    if ell_max >= 6:
        s6 = bin_sums((A0 * np.conj(A["A6"])).real, bidx, w, nb)
        p6 = p6_combination(s0, s2, s4, s6, nmodes, norm)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = ksum / nmodes
    return Multipoles(kmean, nmodes, p0, p2, p4, s0, s2, s4, norm,
                      modes=A if return_modes else None, p6=p6, sum6=s6)
