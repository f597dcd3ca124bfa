"""Particle-to-mesh assignment of F = w (n - alpha n_s) (oracle; FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Sec. 4 places galaxies and randoms on a cubic mesh of side L_b by Cloud-in-Cell to
obtain F(r) of Eq. (1).  The mesh holds cell sums (no division by the cell volume):
F_node = sum_gal w W(u - node) - alpha sum_ran w W(u - node), u = (x - box_min)/H,
H = L/N, indices periodic mod N.  W is the separable kernel
  NGP: 1 at the nearest node,
  CIC: 1 - |d| on the two bracketing nodes,
  TSC: 3/4 - d^2 at the nearest node, (1/2)(1/2 -+ d)^2 at its two neighbours.
The interlaced mesh has its nodes at box_min + (i + 1/2) H, i.e. u -> u - 1/2.

Pinned by: NGP on nodes equals the direct sum (tests/test_oracle_pins.py), the
closed-form Poisson shot-noise shapes of CIC and TSC, and mass conservation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

ORDER = {"ngp": 1, "cic": 2, "tsc": 3}


def _stencil(u: np.ndarray, kind: str):
    """Per-axis (node offsets, weights) for grid coordinates u (FP64)."""
    if kind == "ngp":
        i = np.floor(u + 0.5)
        return [(i, np.ones_like(u))]
    if kind == "cic":
        i = np.floor(u)
        d = u - i
        return [(i, 1.0 - d), (i + 1.0, d)]
    if kind == "tsc":
        i = np.floor(u + 0.5)
        d = u - i
        return [(i - 1.0, 0.5 * (0.5 - d) ** 2), (i, 0.75 - d * d), (i + 1.0, 0.5 * (0.5 + d) ** 2)]
    raise ValueError(kind)


def _deposit(mesh_flat, pos, w, box_min, H, n, kind, shift, chunk=4_000_000):
    for s in range(0, pos.shape[0], chunk):
        p = pos[s:s + chunk].astype(np.float64)
        ww = w[s:s + chunk].astype(np.float64)
        u = (p - np.asarray(box_min, dtype=np.float64)) / H - shift
        st = [_stencil(u[:, d], kind) for d in range(3)]
        for ix, wx in st[0]:
            jx = np.mod(ix, n).astype(np.int64)
            for iy, wy in st[1]:
                jy = np.mod(iy, n).astype(np.int64)
                wxy = ww * wx * wy
                for iz, wz in st[2]:
                    jz = np.mod(iz, n).astype(np.int64)
                    flat = (jx * n + jy) * n + jz
                    mesh_flat += np.bincount(flat, weights=wxy * wz, minlength=n ** 3)


_CLIB = None


def _clib():
    """The plain-C loop of oracle/c/deposit.c (same definitions), if built."""
    global _CLIB
    if _CLIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")
        if not os.path.exists(path):
            return None
        lib = ctypes.CDLL(path)
        f = lib.oracle_deposit
        f.restype = None
        f.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
        _CLIB = lib
    return _CLIB


def _deposit_c(lib, mesh_flat, cat, w, box_min, H, n, kind, shift):
    x = np.ascontiguousarray(cat.x, dtype=np.float32)
    y = np.ascontiguousarray(cat.y, dtype=np.float32)
    z = np.ascontiguousarray(cat.z, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    bm = np.ascontiguousarray(box_min, dtype=np.float64)
    lib.oracle_deposit(x.ctypes.data, y.ctypes.data, z.ctypes.data, w.ctypes.data, x.shape[0], bm.ctypes.data,
                       float(H), int(n), ORDER[kind], float(shift), mesh_flat.ctypes.data)


def assign_mesh(gal, ran, alpha: float, box_min, box_len: float, n: int, kind: str = "cic",
                interlaced: bool = False, impl: str = "auto") -> np.ndarray:
    """FP64 mesh (n, n, n), x-major (z fastest), of F = w_gal - alpha w_ran cell sums.

    ``interlaced`` gives the second mesh, whose nodes sit at +H/2 on every axis.
    ``impl``: "numpy", "c" (oracle/c/deposit.c, built by oracle/cbuild.py) or "auto"
    (C when built).  Both follow the definitions in the module header.
    """
    H = box_len / n
    shift = 0.5 if interlaced else 0.0
    flat = np.zeros(n ** 3, dtype=np.float64)
    lib = _clib() if impl in ("auto", "c") else None
    if impl == "c" and lib is None:
        raise RuntimeError("oracle C helper not built (python oracle/cbuild.py)")
    wr = -alpha * ran.w.astype(np.float64)
    if lib is not None:
        _deposit_c(lib, flat, gal, gal.w.astype(np.float64), box_min, H, n, kind, shift)
        _deposit_c(lib, flat, ran, wr, box_min, H, n, kind, shift)
    else:
        _deposit(flat, gal.positions(), gal.w, box_min, H, n, kind, shift)
        _deposit(flat, ran.positions(), wr, box_min, H, n, kind, shift)
    return flat.reshape(n, n, n)
