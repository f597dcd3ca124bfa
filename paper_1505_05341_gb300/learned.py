"""Learned aliasing/window correction: training pairs, GPU training, evaluation.

The pairs come from the estimator itself.  Each seeded config-1-style mock (clustered
Zel'dovich + RSD galaxies in a 500 Mpc/h cube centred on (600, 600, 600), observer at
the origin, randoms 5 N_g) is measured on a coarse 128^3 CIC mesh without
interlacing, in shells of 0.01 h/Mpc up to 0.80 h/Mpc (below the coarse Nyquist
frequency).  Its target is one of:
  * the fine 512^3 TSC mesh with interlacing (N_g uniform in 2e5-2e6), whose shells
    see the same modes;
  * on small cases (N_g uniform in 2e4-6e4), the direct galaxy sum of Sec. 4
    (ys_sum_gal) at the coarse lattice's own modes: no mesh, window or aliasing.
The network (ys_mlp, include/ystat.h) learns the scaled residual of each shell,
trained on targets divided by their common RMS (the scale is folded back into the
output layer afterwards, so the saved network predicts the residual itself).  The
three outputs share that one scale: weighting P_2's residual, an order of magnitude
smaller than the others, up to unit RMS made the network fit that residual's
realisation-to-realisation noise, and the held-out P_2 residual grew (rms 6.1e-3 ->
7.0e-3 on a short direct-sum training) instead of falling.
Training, inference and the correction all run in the library's kernels -- this
module only sequences the calls.

    python -m paper_1505_05341_gb300.learned --train 2000 --direct 200 --heldout 200 --out weights.npz
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
DIRECT_SEEDS = 30_000          # small mocks with direct-sum targets (training)
DIRECT_HELDOUT_SEEDS = 40_000  # and held out
DIRECT_N_GAL = (20_000, 60_000)
# parameter layout: W1 b1 W2 b2 W3 b3 W4[3][64] b4[3]; the output layer starts here
W4_OFFSET = 5 * 64 + 64 + 64 * 64 + 64 + 64 * 64 + 64
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

    def direct_rows(self, seeds):
        """Device rows (len(seeds), stride) of the coarse mesh and of the direct galaxy
        sum at the coarse lattice's modes, for small mocks (N_g in DIRECT_N_GAL)."""
        import torch
        import synth.gpu as sg
        n = len(seeds)
        out_c = torch.zeros((n, self.stride), dtype=torch.float64, device="cuda")
        out_d = torch.zeros((n, self.stride), dtype=torch.float64, device="cuda")
        for i, seed in enumerate(seeds):
            ng, nr = sg.mock_sizes(seed, DIRECT_N_GAL)
            gal, ran, _ = sg.zeldovich_cube(ng, nr, seed)
            self.coarse.assign(gal, ran)
            self.coarse.measure_async(out_c[i])
            d = ystat.sum_gal(COARSE["n_mesh"], BOX_MIN, BOX_LEN, gal, ran, observer=OBSERVER, dk=DK,
                              n_bins=N_BINS)
            out_d[i] = torch.from_numpy(np.concatenate([d.k, d.n_modes, d.p0, d.p2, d.p4,
                                                        [d.alpha, d.norm_I, d.shot_noise, 0.0, 0.0]]))
            del gal, ran
        torch.cuda.synchronize()
        return out_c, out_d

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


def target_scales(T):
    """The targets' common RMS, as a scale for each of the three outputs."""
    import torch
    return torch.sqrt(torch.mean(T.double() ** 2)).clamp_min(1e-12).float().repeat(3)


def fold_scales(mlp, scales):
    """A network trained on targets / scales predicts the residual itself once its
    output layer (W4 row l and b4[l]) is multiplied by scales[l]."""
    w, m, v, t = mlp.state()
    sc = scales.cpu().numpy().astype(np.float32)
    for l in range(3):
        w[W4_OFFSET + 64 * l:W4_OFFSET + 64 * (l + 1)] *= sc[l]
        w[W4_OFFSET + 3 * 64 + l] *= sc[l]
    mlp.set_state(w, m, v, t)


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
    ap.add_argument("--direct", type=int, default=200, help="small mocks with direct-sum targets")
    ap.add_argument("--direct-heldout", type=int, default=20)
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
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    dr_c = dr_d = dh_c = dh_d = None
    if a.direct > 0:
        dr_c, dr_d = pm.direct_rows(list(range(DIRECT_SEEDS, DIRECT_SEEDS + a.direct)))
    if a.direct_heldout > 0:
        dh_c, dh_d = pm.direct_rows(list(range(DIRECT_HELDOUT_SEEDS, DIRECT_HELDOUT_SEEDS + a.direct_heldout)))
    pm.close()
    t_direct = time.perf_counter() - t0
    X, T, _, m = features(tr_c, tr_f)
    m_direct = 0
    if dr_c is not None:
        Xd, Td, _, m_direct = features(dr_c, dr_d)
        X, T = torch.cat([X, Xd]), torch.cat([T, Td])
    scales = target_scales(T)
    mlp = ystat.Mlp(init_params(a.seed))
    t1 = time.perf_counter()
    hist = train(mlp, X, (T / scales).contiguous(), a.steps, a.lr, a.lr_final, log_every=max(1, a.steps // 20))
    fold_scales(mlp, scales)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    before, after = evaluate(mlp, ho_c, ho_f)
    tr_before, tr_after = evaluate(mlp, tr_c, tr_f)
    d_before = d_after = None
    if dh_c is not None:
        d_before, d_after = evaluate(mlp, dh_c, dh_d)
    meta = dict(train_seeds=[TRAIN_SEEDS, TRAIN_SEEDS + a.train - 1],
                heldout_seeds=[HELDOUT_SEEDS, HELDOUT_SEEDS + a.heldout - 1],
                direct_seeds=[DIRECT_SEEDS, DIRECT_SEEDS + a.direct - 1] if a.direct else None,
                direct_heldout_seeds=([DIRECT_HELDOUT_SEEDS, DIRECT_HELDOUT_SEEDS + a.direct_heldout - 1]
                                      if a.direct_heldout else None),
                direct_n_gal=list(DIRECT_N_GAL), rows=m, direct_rows=m_direct, steps=a.steps,
                lr=a.lr, lr_final=a.lr_final, init_seed=a.seed, loss=hist, pair_seconds=t_pairs,
                direct_seconds=t_direct, train_seconds=t_train, target_scales=scales.cpu().tolist(),
                heldout_before=before, heldout_after=after, train_before=tr_before, train_after=tr_after,
                direct_heldout_before=d_before, direct_heldout_after=d_after, coarse=COARSE, fine=FINE, dk=DK,
                n_bins=N_BINS,
                note="Adam moments are those of the scaled-target training; the saved parameters "
                     "have the scales folded into the output layer")
    save(a.out, mlp, meta)
    print(json.dumps({k: meta[k] for k in ("rows", "direct_rows", "pair_seconds", "direct_seconds",
                                           "train_seconds", "target_scales", "heldout_before",
                                           "heldout_after", "direct_heldout_before", "direct_heldout_after")}))
    print("loss", hist[0], hist[-1])
    mlp.close()
    del torch
    return meta


if __name__ == "__main__":
    main()
