"""GPU kernels of the learned correction against the FP64 reference network.

Forward outputs, gradients and Adam updates are compared with oracle.mlp evaluated
at the same bfloat16-rounded weights and the same float32 inputs; the feature and
correction kernels against oracle.mlp.features_and_targets; and a short training on
pairs produced by the estimator must lower the held-out residual."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_05341_gb300 as ys
    return ys


def _inputs(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, 5)).astype(np.float32)
    X[:, 0] = rng.uniform(0, 1, rows)
    T = (0.3 * rng.standard_normal((rows, 3))).astype(np.float32)
    return X, T


@pytest.mark.parametrize("rows", [1, 63, 64, 65, 1000])
def test_forward_matches_oracle(ys, rows):
    p = ref.init_params(11)
    X, _ = _inputs(rows, rows)
    net = ys.Mlp(p)
    dX = torch.from_numpy(X).cuda()
    dY = torch.empty((rows, 3), dtype=torch.float32, device="cuda")
    net.forward(dX, dY)
    torch.cuda.synchronize()
    Y_ref, _ = ref.forward(ref.bf16_round(p), X.astype(np.float64))
    Y = dY.cpu().numpy().astype(np.float64)
    scale = np.abs(Y_ref).max()
    assert np.abs(Y - Y_ref).max() <= 1e-5 * max(1.0, scale)
    net.close()


@pytest.mark.parametrize("rows", [7, 64, 129, 2000])
def test_gradient_matches_oracle(ys, rows):
    p = ref.init_params(12)
    X, T = _inputs(rows, 100 + rows)
    net = ys.Mlp(p)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    g = torch.empty(ys.MLP_PARAMS, dtype=torch.float32, device="cuda")
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.gradient(dX, dT, d_grad=g, d_sse=sse)
    torch.cuda.synchronize()
    loss_ref, g_ref = ref.loss_and_grad(ref.bf16_round(p), X.astype(np.float64), T.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(sse.item()) / (3 * rows) - loss_ref) <= 1e-5 * loss_ref
    # per layer: worst element within 1e-3 of that layer's largest gradient
    off = 0
    for fan_in, fan_out in ref.LAYERS:
        for size in (fan_in * fan_out, fan_out):
            a, b = gg[off:off + size], g_ref[off:off + size]
            assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max(), (off, size)
            off += size
    assert np.linalg.norm(gg - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    net.close()


def test_adam_steps_match_oracle(ys):
    p = ref.init_params(13)
    X, T = _inputs(300, 7)
    net = ys.Mlp(p)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    w = p.astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t in (1, 2, 3):
        net.train_step(dX, dT, 1e-3)
        # the oracle takes the step from the gradient at the same bfloat16 weights
        _, g = ref.loss_and_grad(ref.bf16_round(w.astype(np.float32)), X.astype(np.float64), T.astype(np.float64))
        w, m, v = ref.adam_step(w, g, m, v, t, 1e-3)
        w_gpu, m_gpu, v_gpu, step = net.state()
        assert step == t
        # Adam's step is about lr g / |g|, so where |g| is near float32 noise the
        # direction is not determined; elsewhere the two steps agree closely
        sure = np.abs(g) > 1e-5 * np.abs(g).max()
        assert sure.mean() > 0.99
        assert np.abs(w_gpu - w)[sure].max() <= 2e-5, t
        assert np.abs(w_gpu - w).max() <= 2.1e-3 * t
        assert np.abs(m_gpu - m).max() <= 1e-3 * np.abs(m).max()
        w = w_gpu.astype(np.float64)  # follow the device weights (float32 rounding)
    net.close()


def test_state_roundtrip(ys):
    p = ref.init_params(14)
    net = ys.Mlp(p)
    rng = np.random.default_rng(0)
    m = rng.standard_normal(ys.MLP_PARAMS).astype(np.float32)
    v = rng.uniform(0, 1, ys.MLP_PARAMS).astype(np.float32)
    net.set_state(p, m, v, 17)
    w2, m2, v2, t = net.state()
    assert t == 17 and np.array_equal(w2, p) and np.array_equal(m2, m) and np.array_equal(v2, v)
    net.close()


def _synthetic_rows(n_cat, n_bins, seed):
    """Result rows with plausible multipoles, some empty, negative-D and NaN shells."""
    rng = np.random.default_rng(seed)
    stride = 5 * n_bins + 5
    rows = np.zeros((n_cat, stride))
    fine = np.zeros((n_cat, stride))
    for c in range(n_cat):
        k = (np.arange(n_bins) + 0.5) * 0.01
        nm = rng.integers(0, 50, n_bins).astype(float)
        p_sn = rng.uniform(50, 500)
        p0 = rng.uniform(-0.5, 30, n_bins) * p_sn
        p0[rng.integers(0, n_bins)] = -2 * p_sn        # D < 0
        p2 = rng.standard_normal(n_bins) * p_sn
        p4 = rng.standard_normal(n_bins) * p_sn
        p2[rng.integers(0, n_bins)] = np.nan
        rows[c, :n_bins] = k
        rows[c, n_bins:2 * n_bins] = nm
        rows[c, 2 * n_bins:3 * n_bins] = p0
        rows[c, 3 * n_bins:4 * n_bins] = p2
        rows[c, 4 * n_bins:5 * n_bins] = p4
        rows[c, 5 * n_bins:] = [0.2, 1e-3, p_sn, 0, 0]
        fine[c] = rows[c]
        fine[c, 2 * n_bins:5 * n_bins] += rng.standard_normal(3 * n_bins) * 0.1 * p_sn
    return rows, fine


def test_features_and_correction_match_oracle(ys):
    n_cat, nb, k_nyq = 5, 37, 0.8
    rows, fine = _synthetic_rows(n_cat, nb, 3)
    d_rows = torch.from_numpy(rows).cuda()
    d_fine = torch.from_numpy(fine).cuda()
    n = n_cat * nb
    X = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    T = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ys.Mlp.features(d_rows, nb, k_nyq, X, src, cnt, d_fine_rows=d_fine, d_t=T)
    torch.cuda.synchronize()
    m = int(cnt.item())
    src_h = src[:m].cpu().numpy()
    X_h, T_h = X[:m].cpu().numpy(), T[:m].cpu().numpy()
    want_idx, want_X, want_T = [], [], []
    for c in range(n_cat):
        r, f = rows[c], fine[c]
        idx, Xr, Tr = ref.features_and_targets(r[:nb], r[nb:2 * nb], r[2 * nb:3 * nb], r[3 * nb:4 * nb],
                                               r[4 * nb:5 * nb], r[5 * nb + 2], k_nyq,
                                               fine=(f[2 * nb:3 * nb], f[3 * nb:4 * nb], f[4 * nb:5 * nb]))
        want_idx += list(c * nb + idx)
        want_X.append(Xr)
        want_T.append(Tr)
    want_X, want_T = np.concatenate(want_X), np.concatenate(want_T)
    assert sorted(src_h.tolist()) == sorted(want_idx)          # same set of shells, order free
    order = np.argsort(src_h)
    np.testing.assert_allclose(X_h[order], want_X, rtol=2e-7, atol=1e-7)
    np.testing.assert_allclose(T_h[order], want_T, rtol=2e-7, atol=1e-7)

    # correction: rows + D y, y = network at the bfloat16 weights on the float32 features
    p = ref.init_params(15)
    net = ys.Mlp(p)
    out = torch.empty_like(d_rows)
    net.correct(d_rows, nb, k_nyq, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = rows.copy()
    y, _ = ref.forward(ref.bf16_round(p), X_h[order].astype(np.float64))
    for j, sidx in enumerate(sorted(want_idx)):
        c, b = divmod(sidx, nb)
        D = rows[c, 2 * nb + b] + rows[c, 5 * nb + 2]
        for l in range(3):
            want[c, (2 + l) * nb + b] += D * y[j, l]
    same = np.isnan(want) & np.isnan(got)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    # the increments D y carry the float32 error of the network's outputs
    d_got = np.where(same, 0, got - rows)
    d_want = np.where(same, 0, want - rows)
    D_max = np.nanmax(np.abs(rows[:, 2 * nb:3 * nb] + rows[:, 5 * nb + 2][:, None]))
    assert np.abs(d_got - d_want).max() <= 1e-5 * D_max * max(1.0, np.abs(y).max())
    assert np.array_equal(np.where(d_want == 0, 1, 0), np.where(d_got == 0, 1, 0))
    # in place gives the same
    net.correct(d_rows, nb, k_nyq, d_rows)
    torch.cuda.synchronize()
    inplace = d_rows.cpu().numpy()
    assert np.array_equal(np.nan_to_num(inplace, nan=7.0), np.nan_to_num(got, nan=7.0))
    net.close()


def test_training_lowers_heldout_residual(ys):
    """A short training on 24 estimator-made pairs (N_g 2e5-4e5) must cut the held-out
    residual of the coarse monopole against the fine mesh."""
    from paper_1505_05341_gb300 import learned
    pm = learned.PairMaker(max_particles=2_400_000, n_gal_range=(200_000, 400_000))
    tr_c, tr_f = pm.rows(list(range(50_000, 50_024)))
    ho_c, ho_f = pm.rows(list(range(60_000, 60_008)))
    pm.close()
    X, T, _, m = learned.features(tr_c, tr_f)
    assert m > 20 * learned.N_BINS
    net = ys.Mlp(learned.init_params(0))
    hist = learned.train(net, X, T, 800, lr=1e-3, lr_final=1e-4, log_every=100)
    assert hist[-1][1] < 0.2 * hist[0][1]
    before, after = learned.evaluate(net, ho_c, ho_f)
    print("held-out residual before", before, "after", after)
    assert after["rms0"] < 0.5 * before["rms0"]
    net.close()


def test_folded_scales_reproduce_scaled_outputs(ys):
    """A network trained on targets / s predicts the residual once s is folded into its
    output layer: the folded outputs equal the unfolded ones times s."""
    from paper_1505_05341_gb300 import learned
    p = ref.init_params(21)
    X, _ = _inputs(300, 21)
    dX = torch.from_numpy(X).cuda()
    net = ys.Mlp(p)
    y0 = torch.empty((300, 3), dtype=torch.float32, device="cuda")
    net.forward(dX, y0)
    s = torch.tensor([0.08, 0.0065, 0.075], dtype=torch.float32)
    learned.fold_scales(net, s)
    y1 = torch.empty_like(y0)
    net.forward(dX, y1)
    torch.cuda.synchronize()
    want = y0.cpu().numpy() * s.numpy()
    got = y1.cpu().numpy()
    # the kernels use bfloat16 weights: folding re-rounds the output layer
    assert np.abs(got - want).max() <= 1e-2 * np.abs(want).max()
    net.close()


def test_direct_sum_targets_train_the_correction(ys):
    """Pairs with the direct galaxy sum (Sec. 4) as target, on small mocks: a short
    training on 12 of them must cut the held-out residual of the coarse monopole and
    hexadecapole against the direct sum."""
    from paper_1505_05341_gb300 import learned
    pm = learned.PairMaker(max_particles=400_000)
    old = learned.DIRECT_N_GAL
    learned.DIRECT_N_GAL = (20_000, 30_000)
    try:
        tr_c, tr_d = pm.direct_rows(list(range(70_000, 70_012)))
        ho_c, ho_d = pm.direct_rows(list(range(71_000, 71_004)))
    finally:
        learned.DIRECT_N_GAL = old
    pm.close()
    X, T, _, m = learned.features(tr_c, tr_d)
    assert m > 10 * learned.N_BINS
    scales = learned.target_scales(T)
    net = ys.Mlp(learned.init_params(0))
    learned.train(net, X, (T / scales).contiguous(), 800, lr=1e-3, lr_final=1e-4)
    learned.fold_scales(net, scales)
    before, after = learned.evaluate(net, ho_c, ho_d)
    print("direct-sum targets: held-out residual before", before, "after", after)
    assert after["rms0"] < 0.7 * before["rms0"]
    assert after["rms4"] < 0.7 * before["rms4"]
    net.close()
