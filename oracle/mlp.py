"""FP64 reference of the learned aliasing/window correction network (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Not part of the paper: the coarse-mesh multipoles P_l(k) carry aliasing and window
residuals (Sec. 4 notes aliasing as the source of the sum-grid deviation); a small
network maps per-shell features of a coarse measurement to the residual against a
fine mesh.  Architecture 5 -> 64 -> 64 -> 64 -> 3, GELU (exact erf form) after each
hidden layer, linear output; loss = mean squared error over rows and outputs.

Parameter vector layout (float, row-major weights W[out][in]):
  W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[3][64] b4[3]

Features of one shell of a coarse measurement, with D = P_0 + P_SN the monopole
before shot-noise subtraction and P_SN = S/I:
  x = [k / k_N, ln(D / P_SN), P_2 / D, P_4 / D, P_SN / D];
targets t_l = (P_l^fine - P_l^coarse) / D; the correction adds D y_l to P_l.

Pinned by: central finite differences of the loss (tests/test_oracle_mlp.py), GELU
against its erf definition evaluated with math.erf, the first Adam step's closed
form (each parameter moves by lr sign(g)), and a hand-worked feature row.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

LAYERS = [(5, 64), (64, 64), (64, 64), (64, 3)]
N_PARAMS = sum(i * o + o for i, o in LAYERS)


def unpack(params):
    """List of (W [out, in], b [out]) views into the flat parameter vector."""
    out = []
    off = 0
    for i, o in LAYERS:
        W = params[off:off + i * o].reshape(o, i)
        off += i * o
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + scipy.special.erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + scipy.special.erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(params, X):
    """Outputs (rows x 3) and the per-layer cache (pre-activations, inputs)."""
    layers = unpack(np.asarray(params, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h, cache


def loss_and_grad(params, X, T):
    """MSE loss = mean over rows and outputs of (y - t)^2, and its gradient."""
    params = np.asarray(params, dtype=np.float64)
    Y, cache = forward(params, X)
    T = np.asarray(T, dtype=np.float64)
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    layers = unpack(params)
    grads = []
    d = 2.0 * (Y - T) / n
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        h, z = cache[li]
        if li < len(layers) - 1:
            d = d * gelu_grad(z)
        grads.append((d.T @ h, d.sum(axis=0)))
        d = d @ W
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (float32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in LAYERS:
        bound = 1.0 / math.sqrt(i)
        parts.append(rng.uniform(-bound, bound, size=i * o))
        parts.append(rng.uniform(-bound, bound, size=o))
    return np.concatenate(parts).astype(np.float32)


def adam_step(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, bias-corrected); t is the new step count
    (1 for the first step).  Returns (params, m, v)."""
    params, grad = np.asarray(params, np.float64), np.asarray(grad, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * grad
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features_and_targets(k_mean, n_modes, p0, p2, p4, p_sn, k_nyq, fine=None):
    """Feature rows (and target rows if fine = (P0, P2, P4) of the fine mesh) of the
    shells that have modes, finite multipoles and D > 0.  Returns (shell indices,
    X [n, 5], T [n, 3] or None)."""
    k_mean, n_modes, p0, p2, p4 = (np.asarray(a, np.float64) for a in (k_mean, n_modes, p0, p2, p4))
    D = p0 + p_sn
    ok = (n_modes > 0) & np.isfinite(p0) & np.isfinite(p2) & np.isfinite(p4) & (D > 0) & (p_sn > 0)
    if fine is not None:
        f0, f2, f4 = (np.asarray(a, np.float64) for a in fine)
        ok &= np.isfinite(f0) & np.isfinite(f2) & np.isfinite(f4)
    idx = np.nonzero(ok)[0]
    d = D[idx]
    X = np.stack([k_mean[idx] / k_nyq, np.log(d / p_sn), p2[idx] / d, p4[idx] / d, p_sn / d], axis=1)
    T = None
    if fine is not None:
        T = np.stack([(f0[idx] - p0[idx]) / d, (f2[idx] - p2[idx]) / d, (f4[idx] - p4[idx]) / d], axis=1)
    return idx, X, T
