"""Catalogue sums: alpha, the normalisation I and the shot noise S (oracle; FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Eq. (1): F(r) = w(r) [n(r) - alpha n_s(r)] / I^(1/2), with alpha normalising the
weighted randoms to the weighted galaxies and I = int w^2 nbar^2 dr.
Eq. (3): P_l^noise = (1 + alpha) int nbar w^2 L_l dr.

Discrete readings (the paper gives only the integrals):
* alpha = sum_gal w / sum_ran w.
* I = alpha * sum_ran w^2 nbar  (the random catalogue samples nbar with density
  nbar/alpha, so this sum estimates int w^2 nbar^2 dr).
* S = sum_gal w^2 + alpha^2 sum_ran w^2 (the self-pair term of the direct sum; its
  expectation is (1 + alpha) int nbar w^2 dr).

Pinned by: the closed form S/I = (1 + alpha)/nbar for unit weights and uniform nbar
(tests/test_oracle_pins.py::test_norm_closed_form) and the Poisson shot-noise test.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Norm:
    alpha: float
    I: float
    S: float
    sum_w_gal: float
    sum_w_ran: float


def catalog_sums(gal, ran, alpha: float | None = None) -> Norm:
    wg = gal.w.astype(np.float64)
    wr = ran.w.astype(np.float64)
    nr = ran.nbar.astype(np.float64)
    swg = float(np.sum(wg))
    swr = float(np.sum(wr))
    a = swg / swr if alpha is None or alpha < 0 else float(alpha)
    I = a * float(np.sum(wr * wr * nr))
    S = float(np.sum(wg * wg)) + a * a * float(np.sum(wr * wr))
    return Norm(a, I, S, swg, swr)
