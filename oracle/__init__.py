"""FP64 CPU oracle for the FFT-based Yamamoto multipole estimator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.  The
GPU library never imports, links or calls this package, and this package shares no
code with it: the two only share the seeded input generators in ``synth``.

Three independent routes to the same estimator (Sec. 4 of the paper):

* ``estimator.fft_multipoles`` -- the FFT-based method: mesh assignment, the 1 + 6
  + 15 line-of-sight weighted fields of Eqs. (11) and (13), one FP64 real-to-complex
  FFT per field, A_2 and A_4 assembled literally from Eqs. (10) and (12), the
  Legendre combinations of Eqs. (6)-(8) and |k|-shell averages.
* ``direct.sum_grid`` -- the same A_n(k) of Eq. (5) as a plain sum over mesh nodes
  with (k.r)^n evaluated per node ("sum-grid").
* ``direct.sum_gal`` -- Eq. (5) as a plain sum over galaxies and randoms ("sum-gal").

Parity status of each function is stated in its module header.
"""
from .normalization import catalog_sums, Norm
from .binning import BinSpec, half_modes, mode_bins
from .assignment import assign_mesh
from .terms import A2_TERMS, A4_TERMS
from .estimator import fft_multipoles, Multipoles
from .direct import sum_gal, sum_grid

__all__ = ["catalog_sums", "Norm", "BinSpec", "half_modes", "mode_bins", "assign_mesh",
           "A2_TERMS", "A4_TERMS", "fft_multipoles", "Multipoles", "sum_gal", "sum_grid"]
