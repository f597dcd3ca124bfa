"""Learned aliasing/window correction: training pairs, GPU training, evaluation.

The pairs come from the estimator itself: each seeded config-1-style mock (clustered
Zel'dovich + RSD galaxies in a 500 Mpc/h cube centred on (600, 600, 600), observer at
the origin, N_g uniform in 2e5-2e6, randoms 5 N_g) is measured on a coarse 128^3 CIC
mesh without interlacing and on a fine 512^3 TSC mesh with interlacing, in shells of
0.01 h/Mpc up to 0.80 h/Mpc (below the coarse Nyquist frequency, so both meshes see
the same modes in every shell).  The network (ys_mlp, include/ystat.h) learns the
scaled residual of each shell; training, inference and the correction all run in
the library's kernels -- this module only sequences the calls.

    python -m paper_1505_05341_gb300.learned --train 2000 --heldout 200 --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import ystat

BOX_MIN = (350.0, 350.0, 350.0)
BOX_LEN = 500.0
OBSERVER = (0.0, 0.0, 0.0)
DK = 0.01
N_BINS = 80
COARSE = dict(n_mesh=128, assign="cic", interlace=False)
FINE = dict(n_mesh=512, assign="tsc", interlace=True)
K_NYQ = math.pi * COARSE["n_mesh"] / BOX_LEN
TRAIN_SEEDS = 10_000
HELDOUT_SEEDS = 20_000
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "correction_128cic_512tsc.npz")


def init_params(seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((5, 64), (64, 64), (64, 64), (64, 3)):
        bound = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_in * fan_out))
        parts.append(rng.uniform(-bound, bound, size=fan_out))
    return np.concatenate(parts).astype(np.float32)


class PairMaker:
    """Coarse and fine plans for the mock geometry; ``rows`` measures mocks on both."""

    def __init__(self, max_particles=12_000_000, n_gal_range=(200_000, 2_000_000), stream=None):
        common = dict(box_min=BOX_MIN, box_len=BOX_LEN, observer=OBSERVER, dk=DK, n_bins=N_BINS,
                      max_particles=max_particles, stream=stream)
        self.coarse = ystat.Plan(**COARSE, **common)
        self.fine = ystat.Plan(**FINE, **common)
        self.stride = 5 * N_BINS + 5
        self.n_gal_range = n_gal_range

    def mock(self, seed):
        import synth.gpu as sg
        ng, nr = sg.mock_sizes(seed, self.n_gal_range)
        return sg.zeldovich_cube(ng, nr, seed)

    def rows(self, seeds, fine=True):
        """Device float64 result rows (len(seeds), stride) of the coarse (and fine) mesh."""
        import torch
        n = len(seeds)
        out_c = torch.zeros((n, self.stride), dtype=torch.float64, device="cuda")
        out_f = torch.zeros((n, self.stride), dtype=torch.float64, device="cuda") if fine else None
        for i, seed in enumerate(seeds):
            gal, ran, _ = self.mock(seed)
            self.coarse.assign(gal, ran)
            self.coarse.measure_async(out_c[i])
            if fine:
                self.fine.assign(gal, ran)
                self.fine.measure_async(out_f[i])
            del gal, ran
        torch.cuda.synchronize()
        return out_c, out_f

    def close(self):
        self.coarse.close()
        self.fine.close()


def features(rows, fine_rows=None):
    """(X, T or None, src, count) device tensors for the shells of ``rows``."""
    import torch
    n = rows.shape[0] * N_BINS
    X = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    T = torch.empty((n, 3), dtype=torch.float32, device="cuda") if fine_rows is not None else None
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ystat.Mlp.features(rows, N_BINS, K_NYQ, X, src, cnt, d_fine_rows=fine_rows, d_t=T)
    m = int(cnt.item())
    return X[:m], (T[:m] if T is not None else None), src[:m], m


def train(mlp, X, T, steps, lr=1e-3, lr_final=None, log_every=0):
    """Full-batch Adam on (X, T); the learning rate decays geometrically from lr to
    lr_final (default lr: constant).  Returns the loss after each logged step."""
    import torch
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    rows = X.shape[0]
    lr_final = lr if lr_final is None else lr_final
    hist = []
    for s in range(steps):
        rate = lr * (lr_final / lr) ** (s / max(1, steps - 1))
        mlp.train_step(X, T, rate, d_sse=sse)
        if log_every and (s % log_every == 0 or s == steps - 1):
            hist.append((s, float(sse.item()) / (3 * rows)))
    torch.cuda.synchronize()
    return hist


def residual_stats(rows, fine_rows):
    """RMS and max over the shells of |P_l - P_l^fine| / D for l = 0, 2, 4 (host)."""
    a = rows.cpu().numpy()
    f = fine_rows.cpu().numpy()
    nb = N_BINS
    out = {}
    nm = a[:, nb:2 * nb]
    D = a[:, 2 * nb:3 * nb] + a[:, 5 * nb + 2][:, None]
    ok = (nm > 0) & (D > 0)
    for j, ell in enumerate((0, 2, 4)):
        e = (a[:, (2 + j) * nb:(3 + j) * nb] - f[:, (2 + j) * nb:(3 + j) * nb]) / np.where(ok, D, 1.0)
        e = e[ok]
        out[f"rms{ell}"] = float(np.sqrt(np.mean(e ** 2)))
        out[f"max{ell}"] = float(np.max(np.abs(e)))
    return out


def evaluate(mlp, coarse_rows, fine_rows):
    """Held-out residuals before and after the correction."""
    import torch
    corr = torch.empty_like(coarse_rows)
    mlp.correct(coarse_rows, N_BINS, K_NYQ, corr)
    torch.cuda.synchronize()
    return residual_stats(coarse_rows, fine_rows), residual_stats(corr, fine_rows)


def save(path, mlp, meta):
    w, m, v, t = mlp.state()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez(path, params=w, adam_m=m, adam_v=v, step=np.int64(t), meta=json.dumps(meta))


def load(path=WEIGHTS):
    """(Mlp with the saved state, metadata dict)."""
    z = np.load(path)
    mlp = ystat.Mlp(z["params"])
    mlp.set_state(z["params"], z["adam_m"], z["adam_v"], int(z["step"]))
    return mlp, json.loads(str(z["meta"]))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args(argv)
    import torch
    t0 = time.perf_counter()
    pm = PairMaker()
    tr_c, tr_f = pm.rows(list(range(TRAIN_SEEDS, TRAIN_SEEDS + a.train)))
    ho_c, ho_f = pm.rows(list(range(HELDOUT_SEEDS, HELDOUT_SEEDS + a.heldout)))
    pm.close()
    t_pairs = time.perf_counter() - t0
    X, T, _, m = features(tr_c, tr_f)
    mlp = ystat.Mlp(init_params(a.seed))
    t1 = time.perf_counter()
    hist = train(mlp, X, T, a.steps, a.lr, a.lr_final, log_every=max(1, a.steps // 20))
    t_train = time.perf_counter() - t1
    before, after = evaluate(mlp, ho_c, ho_f)
    tr_before, tr_after = evaluate(mlp, tr_c, tr_f)
    meta = dict(train_seeds=[TRAIN_SEEDS, TRAIN_SEEDS + a.train - 1],
                heldout_seeds=[HELDOUT_SEEDS, HELDOUT_SEEDS + a.heldout - 1], rows=m, steps=a.steps,
                lr=a.lr, lr_final=a.lr_final, init_seed=a.seed, loss=hist, pair_seconds=t_pairs,
                train_seconds=t_train, heldout_before=before, heldout_after=after, train_before=tr_before,
                train_after=tr_after, coarse=COARSE, fine=FINE, dk=DK, n_bins=N_BINS)
    save(a.out, mlp, meta)
    print(json.dumps({k: meta[k] for k in ("rows", "pair_seconds", "train_seconds", "heldout_before",
                                           "heldout_after", "train_before", "train_after")}))
    print("loss", hist[0], hist[-1])
    mlp.close()
    del torch
    return meta


if __name__ == "__main__":
    main()
