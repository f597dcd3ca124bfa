"""k-mode enumeration and |k|-shell binning (oracle; FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The shell average int dOmega_k / 4pi of Eqs. (6)-(8) becomes a mean over the grid
modes k = k_F m (k_F = 2 pi / L, m integer) whose |k| falls in the bin.  Readings:

* Only the non-redundant half of k space is visited (Sec. 4 uses Hermitian symmetry):
  the real-to-complex layout m_z in [0, N/2], with weight 2 for 0 < m_z < N/2 and 1
  for m_z = 0, so the weighted count equals the full-grid count.
* A mode enters bin b = floor((|k| - k_min)/dk) when 0 <= b < n_bins, m != 0 and
  |k| < k_Nyquist = k_F N / 2 (every mode on a Nyquist plane is therefore dropped,
  which removes the sign ambiguity of k_i there).
* The reported k of a bin is the weighted mean |k| of its modes; empty bins give NaN.

Pinned by: the weighted count equals a brute-force count over the full grid
(tests/test_oracle_pins.py::test_half_mode_weights).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class BinSpec:
    k_min: float
    dk: float
    n_bins: int

    @staticmethod
    def up_to(k_max: float, dk: float, k_min: float = 0.0) -> "BinSpec":
        return BinSpec(k_min, dk, int(math.ceil((k_max - k_min) / dk - 1e-9)))


def kfund(box_len: float) -> float:
    return 2.0 * math.pi / box_len


def half_modes(n: int):
    """Integer frequencies (mx, my, mz) of the rfftn layout [n, n, n//2+1] as
    broadcastable int64 arrays, and the Hermitian weight array."""
    m = np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)
    mz = np.arange(n // 2 + 1, dtype=np.int64)
    mx = m[:, None, None]
    my = m[None, :, None]
    mzz = mz[None, None, :]
    wz = np.where((mz > 0) & (mz < n // 2), 2.0, 1.0)[None, None, :]
    return mx, my, mzz, wz


def mode_bins(n: int, box_len: float, bins: BinSpec):
    """Bin index per half-grid mode (-1 = not used) and the Hermitian weight."""
    mx, my, mz, wz = half_modes(n)
    m2 = mx * mx + my * my + mz * mz
    kf = kfund(box_len)
    kmag = kf * np.sqrt(m2.astype(np.float64))
    b = np.floor((kmag - bins.k_min) / bins.dk)
    k_nyq = kf * n / 2.0
    ok = (m2 > 0) & (kmag < k_nyq) & (b >= 0) & (b < bins.n_bins)
    bidx = np.where(ok, b, -1).astype(np.int64)
    w = np.broadcast_to(wz, bidx.shape) * (bidx >= 0)
    return bidx, w, kmag


def bin_sums(values, bidx, w, n_bins):
    """Weighted sums of ``values`` per bin."""
    sel = bidx >= 0
    return np.bincount(bidx[sel], weights=(w * values)[sel], minlength=n_bins)[:n_bins]
