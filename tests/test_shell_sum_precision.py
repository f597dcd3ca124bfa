"""Precision of the x stage's shell sums, emulated in float32 on the CPU.

The GPU forms each mode's term (|A_0|^2, Re A_0 A_2^*, Re A_0 A_4^*, times the
Hermitian weight) in float32 and adds it into a float shell bin with a
shared-memory atomic; the atomic returns the value it added to, and Knuth's TwoSum
of (that value, the term) -- computed in float32 -- is the exact rounding error of
the add, which goes into a companion float bin.  The pair is folded into FP64 at
the end.  This test replays that arithmetic on the 4096-shell, 32^3 CIC case
(every shell a single |k|, a few dozen modes, P_4 a small difference of sums)
with the terms taken from the FP64 oracle's transforms rounded to float32, adding
them in a random order as concurrent atomics would, and checks that:

* the compensated pair equals the FP64 sum of the same float32 terms to ~1e-12,
  whatever the order (so the GPU's shell sums behave as FP64 accumulators);
* plain float accumulation of the same terms moves P_4 by more than the 1e-4 bar
  in some shell (the failure the pair removes), and depends on the order;
* with FP64-quality sums, the float32 rounding of the transforms alone keeps every
  P_l within 5e-5 of the oracle -- the part of the budget left for the FFTs;
* the same holds when runs of equal shells among neighbouring modes are first summed
  across lanes with error-carrying adds (the x stage's warp scan) and only then added
  to the bins.
"""
import numpy as np

import oracle
import synth
from oracle.binning import BinSpec, bin_sums, mode_bins
from oracle.estimator import legendre_combination

f32 = np.float32


def _case(seed):
    gal, ran, geo = synth.poisson_cube(5_000, 25_000, seed=seed)
    n = 32
    bins = BinSpec(0.0, np.pi * n / geo.box_len / 4096, 4096)
    ref = oracle.fft_multipoles(gal, ran, geo, n, bins, assign="cic", return_modes=True)
    bidx, w, _ = mode_bins(n, geo.box_len, bins)
    a0, a2, a4 = (ref.modes[k].astype(np.complex64) for k in ("A0", "A2", "A4"))
    wb = np.broadcast_to(w, bidx.shape).astype(f32)
    terms = []
    for a in (a0, a2, a4):   # float32 products, as on the GPU
        t = wb * (a0.real * a.real + a0.imag * a.imag)
        terms.append(t.astype(f32))
    return ref, bidx, w, bins.n_bins, terms


def _twosum_bins(b, v, nb, order):
    s = np.zeros(nb, f32)
    c = np.zeros(nb, f32)
    for i in order:
        k = b[i]
        if k < 0:
            continue
        old, x = s[k], v[i]
        new = f32(old + x)
        xb = f32(new - old)
        c[k] = f32(c[k] + f32(f32(old - f32(new - xb)) + f32(x - xb)))
        s[k] = new
    return s.astype(np.float64) + c.astype(np.float64)


def _plain_bins(b, v, nb, order):
    s = np.zeros(nb, f32)
    for i in order:
        if b[i] >= 0:
            s[b[i]] = f32(s[b[i]] + v[i])
    return s.astype(np.float64)


def _worst(ref, sums, nm, has):
    p = legendre_combination(*sums, nm, ref.norm)
    raw = np.where(has, ref.sum0 / np.where(has, nm, 1) / ref.norm.I, 0)
    out = []
    for g, o in zip(p, (ref.p0, ref.p2, ref.p4)):
        sel = has & (np.abs(o) > 1e-2 * raw)
        out.append(float(np.max(np.abs(g[sel] - o[sel]) / np.abs(o[sel]))))
    return out


def test_compensated_float_bins_equal_fp64_accumulation():
    ref, bidx, w, nb, terms = _case(92)
    b = bidx.ravel()
    nm = ref.n_modes
    has = nm > 0
    exact = [bin_sums(t.astype(np.float64), bidx, np.ones_like(w), nb) for t in terms]
    scale = [bin_sums(np.abs(t.astype(np.float64)), bidx, np.ones_like(w), nb) for t in terms]
    rng = np.random.default_rng(0)
    plain_worst = []
    for rep in range(2):
        order = rng.permutation(b.size)
        comp = [_twosum_bins(b, t.ravel(), nb, order) for t in terms]
        for c, e, s in zip(comp, exact, scale):
            assert np.all(np.abs(c - e) <= 1e-12 * s + 1e-30)
        plain = [_plain_bins(b, t.ravel(), nb, order) for t in terms]
        plain_worst.append(_worst(ref, plain, nm, has)[2])
    # float bins alone break the parity bar for P_4 in this case, and move with the order
    assert max(plain_worst) > 1e-4
    assert plain_worst[0] != plain_worst[1]
    # the float32 transforms with FP64-quality sums stay inside half the bar
    assert max(_worst(ref, exact, nm, has)) < 5e-5


def _two_sum_err(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return f32(f32(a - f32(s - bb)) + f32(b - bb))


def _run_reduced_bins(b, v, nb, chunks, order):
    """The x stage's order of operations: the lanes of one pencil (here a chunk of
    neighbouring modes) first sum each run of equal shells in the segmented suffix
    scan's tree order (offsets 1, 2, 4 within the chunk), carrying every add's exact
    error; the run's first lane then adds the sum to the bin and the carried error
    plus the add's own error to the companion bin."""
    s = np.zeros(nb, f32)
    c = np.zeros(nb, f32)
    for ci in order:
        idx = chunks[ci]
        key = b[idx]
        L = idx.size
        val = v[idx].astype(f32).copy()
        cmp = np.zeros(L, f32)
        end = np.array([j == L - 1 or key[j + 1] != key[j] for j in range(L)])
        d = 1
        while d < L:
            vn, cn, en = val.copy(), cmp.copy(), end.copy()
            for j in range(L):
                if not end[j]:
                    cmp[j] = f32(cmp[j] + f32(cn[j + d] + _two_sum_err(val[j], vn[j + d])))
                    val[j] = f32(val[j] + vn[j + d])
                    end[j] = en[j + d]
            d *= 2
        for j in range(L):
            k = key[j]
            if k >= 0 and (j == 0 or key[j - 1] != k):
                old = s[k]
                s[k] = f32(old + val[j])
                c[k] = f32(c[k] + f32(cmp[j] + _two_sum_err(old, val[j])))
    return s.astype(np.float64) + c.astype(np.float64)


def test_run_reduced_compensated_bins_equal_fp64_accumulation():
    ref, bidx, w, nb, terms = _case(93)
    b = bidx.ravel()
    nchunk = b.size // 8
    chunks = [np.arange(8 * i, 8 * i + 8) for i in range(nchunk)]  # neighbouring modes
    exact = [bin_sums(t.astype(np.float64).ravel()[:8 * nchunk], b[:8 * nchunk], np.ones(8 * nchunk), nb)
             for t in terms]
    scale = [bin_sums(np.abs(t.astype(np.float64)).ravel()[:8 * nchunk], b[:8 * nchunk], np.ones(8 * nchunk), nb)
             for t in terms]
    multi = sum(1 for ch in chunks if np.unique(b[ch][b[ch] >= 0]).size > 1)
    assert multi > 0  # some chunks hold more than one run
    order = np.random.default_rng(1).permutation(nchunk)
    for t, e, sc in zip(terms, exact, scale):
        got = _run_reduced_bins(b, t.ravel(), nb, chunks, order)
        assert np.all(np.abs(got - e) <= 1e-12 * sc + 1e-30)
