"""Device-side (torch CUDA) versions of the seeded catalogue generators, for workloads
with hundreds to thousands of mocks where drawing them with numpy on the host would
dominate.  The recipes are the ones of ``synth.catalogs``; the random streams are
torch's (seeded per catalogue), so the points differ from the numpy generators'.

Like the rest of ``synth`` this holds no arithmetic of the estimator: it only makes
inputs.
"""
from __future__ import annotations

import math

import numpy as np

from .catalogs import Geometry

_LINEAR = dict(amp=2.0e4, k0=0.02, slope=-1.5, kcut=0.5)


def _linear_power(k):
    import torch
    p = _LINEAR["amp"] * (k / _LINEAR["k0"]).clamp_min(1e-30) ** _LINEAR["slope"] * torch.exp(-(k / _LINEAR["kcut"]) ** 2)
    return torch.where(k > 0, p, torch.zeros_like(p))


def displacement(n_grid: int, cell: float, gen, device="cuda"):
    """Zel'dovich displacement psi (3, n^3) of a seeded Gaussian density field with
    P(k) = 2e4 (k/0.02)^-1.5 exp(-(k/0.5)^2) on a periodic grid of spacing ``cell``."""
    import torch
    white = torch.randn((n_grid,) * 3, generator=gen, device=device, dtype=torch.float64)
    wk = torch.fft.rfftn(white)
    kf = 2 * math.pi / (n_grid * cell)
    kx = torch.fft.fftfreq(n_grid, d=1.0 / n_grid, device=device, dtype=torch.float64) * kf
    kz = torch.fft.rfftfreq(n_grid, d=1.0 / n_grid, device=device, dtype=torch.float64) * kf
    KX, KY, KZ = torch.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    dk = wk * torch.sqrt(_linear_power(torch.sqrt(k2)) / cell ** 3)
    k2[0, 0, 0] = 1.0
    psi = [torch.fft.irfftn(1j * K * dk / k2, s=(n_grid,) * 3).reshape(-1) for K in (KX, KY, KZ)]
    return torch.stack(psi)


def zeldovich_cube(n_gal: int, n_ran: int, seed: int, side: float = 500.0, center=(600.0, 600.0, 600.0),
                   f_growth: float = 0.7, n_lattice: int = 128, observer=(0.0, 0.0, 0.0), device="cuda"):
    """Clustered redshift-space galaxies in a periodic cube, drawn on the device: a
    lattice of n_lattice^3 points displaced by the Zel'dovich field, shifted along the
    line of sight by f (psi . r_hat), wrapped into the cube and subsampled without
    replacement to n_gal; n_ran uniform randoms; unit weights; nbar = n_gal / side^3.

    Returns (gal, ran, geometry); gal and ran are tuples (x, y, z, w, nbar) of float32
    device tensors."""
    import torch
    if n_lattice ** 3 < n_gal:
        raise ValueError("n_lattice^3 must be >= n_gal")
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    cell = side / n_lattice
    psi = displacement(n_lattice, cell, gen, device)
    lo = torch.tensor(center, dtype=torch.float64, device=device) - 0.5 * side
    pick = torch.randperm(n_lattice ** 3, generator=gen, device=device)[:n_gal]
    iz = pick % n_lattice
    iy = (pick // n_lattice) % n_lattice
    ix = pick // (n_lattice * n_lattice)
    q = torch.stack([ix, iy, iz]).to(torch.float64) * cell + lo[:, None]
    d = psi[:, pick]
    x = q + d
    rel = x - torch.tensor(observer, dtype=torch.float64, device=device)[:, None]
    rhat = rel / torch.linalg.norm(rel, dim=0, keepdim=True)
    s = x + f_growth * (d * rhat).sum(0, keepdim=True) * rhat
    s = lo[:, None] + torch.remainder(s - lo[:, None], side)
    hi = float(np.nextafter(np.float32(float(lo[0]) + side), np.float32(-np.inf)))
    nbar = n_gal / side ** 3

    def pack(p, n):
        p = p.to(torch.float32)
        p = torch.minimum(p, torch.tensor(hi, dtype=torch.float32, device=device))
        return (p[0].contiguous(), p[1].contiguous(), p[2].contiguous(),
                torch.ones(n, device=device), torch.full((n,), nbar, dtype=torch.float32, device=device))

    r = lo[:, None] + side * torch.rand((3, n_ran), generator=gen, device=device, dtype=torch.float64)
    geo = Geometry(tuple(float(v) for v in lo.tolist()), float(side), tuple(float(v) for v in observer))
    return pack(s, n_gal), pack(r, n_ran), geo


def mock_sizes(seed: int, n_gal_range=(200_000, 2_000_000), ran_factor: int = 5):
    """(n_gal, n_ran) of the config-1-style mock with this seed: n_gal uniform in the
    range (drawn from a numpy generator seeded with seed + 7e6), n_ran = 5 n_gal."""
    rng = np.random.default_rng(seed + 7_000_000)
    n_gal = int(rng.integers(n_gal_range[0], n_gal_range[1] + 1))
    return n_gal, ran_factor * n_gal
