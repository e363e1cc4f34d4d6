"""GPU tests of the surrogate network's kernels against the FP64 oracle.

Bars: GEMM entries within 1e-5 of the float64 product of the same BF16
operands, relative to sum |a||b| (FP32 accumulation); forward outputs within
3 % of the RMS of the standardised output; every gradient entry within 8
standard deviations of its propagated BF16 rounding error (unit roundoff
2^-8, probabilistic error analysis) around the FP64 oracle's value on the same
BF16 weights and FP32 biases.
"""
import math

import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import surrogate
    return surrogate


def bf16_round(a):
    """Round-to-nearest-even of float32 values to bfloat16, returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("a_layout,b_layout", [(0, 0), (0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("M,N,K", [(64, 64, 32), (200, 72, 48), (8, 256, 512), (136, 16, 256)])
def test_gemm_layouts(S, a_layout, b_layout, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A = bf16_round(rng.standard_normal((M, K)))
    B = bf16_round(rng.standard_normal((K, N)))
    want = A @ B
    bound = np.abs(A) @ np.abs(B)
    At = A if a_layout == 0 else A.T
    Bt = B.T if b_layout == 0 else B
    net = S.Surrogate(0)
    try:
        tA = torch.from_numpy(np.ascontiguousarray(At, dtype=np.float32)).to(torch.bfloat16).cuda()
        tB = torch.from_numpy(np.ascontiguousarray(Bt, dtype=np.float32)).to(torch.bfloat16).cuda()
        C = net.gemm_bf16(a_layout, b_layout, M, N, K, tA, tB).cpu().numpy().astype(np.float64)
    finally:
        net.close()
    assert np.all(np.abs(C - want) <= 1e-5 * bound + 1e-6)


def _random_net(S, seed):
    rng = np.random.default_rng(seed)
    net = S.Surrogate(seed)
    p = net.get_params().astype(np.float64)
    P = omlp.unflatten(p)
    P["b1"] = rng.standard_normal(256) * 0.1
    P["b2"] = rng.standard_normal(256) * 0.1
    P["b3"] = rng.standard_normal(256) * 0.1
    P["b4"][:2] = [0.3, -0.2]
    p = omlp.flatten(P)
    net.set_params(p.astype(np.float32))
    shift = np.array([1.0, 4.0, 5.0, 0.0, -2.5, 2.5, 0.25])
    scale = np.array([2.0, 0.5, 0.5, 3.3, 0.66, 0.4, 4.0])
    net.set_maps(shift, scale, 1 << 4, np.array([0.1, -3.0]), np.array([0.2, 1.5]))
    return net, p, (shift, scale, 1 << 4, np.array([0.1, -3.0]), np.array([0.2, 1.5]))


def _raw_inputs(rng, M):
    lo = np.array([0.5, 2.0, 3.0, -0.3, 1e-4, 0.1, 0.01])
    hi = np.array([1.5, 6.0, 7.0, 0.3, 1e-1, 5.0, 0.5])
    x = lo + (hi - lo) * rng.random((M, 7))
    x[:, 4] = 10.0 ** rng.uniform(-4, -1, M)
    return x


def test_forward_matches_oracle(S):
    net, p, (shift, scale, mask, osh, osc) = _random_net(S, 1)
    rng = np.random.default_rng(2)
    x = _raw_inputs(rng, 3000)                                # ragged: 47 x 64 rows - 8
    try:
        y = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    finally:
        net.close()
    pb = bf16_round(p)
    xp = omlp.input_map(x.astype(np.float32).astype(np.float64), shift.astype(np.float32),
                        scale.astype(np.float32), mask)
    yp, _ = omlp.forward(pb, xp)
    want = yp * osc + osh
    # error in standardised output units relative to the output's RMS
    err = np.abs(y - want) / osc / np.sqrt(np.mean(yp ** 2, axis=0))
    assert err.max() < 0.03, err.max()


U_BF16 = 2.0 ** -8       # unit roundoff of BF16 (8 significant bits), round to nearest
REL_F32 = 2.0 ** -18     # FP32 SiLU / SiLU' evaluations (fast exponential) and map arithmetic
K_SIGMA = 8.0            # bar in standard deviations of the propagated rounding error


def _grad_error_sigma(pm, xp, tp, M):
    """Standard deviation of g_gpu - g_oracle for every gradient entry, from a
    probabilistic rounding-error analysis (Higham and Mary, SIAM J. Sci.
    Comput. 2019): each rounding of the kernels -- the mapped input, every SiLU
    activation, dY' and every back-propagated dH to BF16, and the FP32 SiLU /
    SiLU' evaluations -- is an independent error of variance (u |x|)^2 / 3, and
    the variances are carried through the oracle's own intermediates on the
    same BF16 weights and FP32 biases (pm) to first order.  FP32 accumulation
    adds (2^-24)^2 per term and is negligible.  A worst-case bound of the same
    chain, with absolute values, grows by sum_k |W_ik| (about 14) per 256-wide
    layer and would not see a wrong entry."""
    P = omlp.unflatten(pm)
    _, (X, H1, A1, H2, A2, H3, A3, Y) = omlp.forward(pm, xp)
    W2s = [P["W1"] ** 2, P["W2"] ** 2, P["W3"] ** 2, P["W4"] ** 2]
    rnd = lambda x: (U_BF16 * x) ** 2 / 3.0
    acts, Hs = [X, A1, A2, A3], [H1, H2, H3]
    VA, VH = [rnd(X) + (2.0 ** -22) ** 2], []
    for l in range(3):
        VH.append(VA[l] @ W2s[l].T + (REL_F32 * Hs[l]) ** 2)
        sp = omlp.dsilu(Hs[l])                       # silu'
        VA.append(sp ** 2 * VH[l] + rnd(acts[l + 1]) + (REL_F32 * acts[l + 1]) ** 2)
    VY = VA[3] @ W2s[3].T
    R = np.zeros_like(Y)
    R[:, :2] = Y[:, :2] - tp
    dY = R / M
    VdY = np.zeros_like(Y)
    VdY[:, :2] = (VY[:, :2] + rnd(R[:, :2])) / M ** 2
    Wup = [P["W2"], P["W3"], P["W4"]]
    dH, VdH = [None] * 3, [None] * 3
    up, Vup = dY, VdY
    for l in (2, 1, 0):
        G = up @ Wup[l]
        VG = Vup @ W2s[l + 1]
        D = omlp.dsilu(Hs[l])
        s = 1.0 / (1.0 + np.exp(-Hs[l]))
        D2 = s * (1 - s) * (2.0 + Hs[l] * (1 - 2 * s))   # silu''
        VD = D2 ** 2 * VH[l] + (REL_F32 * D) ** 2
        dH[l] = G * D
        VdH[l] = VG * D ** 2 + G ** 2 * VD + rnd(dH[l])
        up, Vup = dH[l], VdH[l]
    lower = [X, A1, A2]
    var = {}
    for l in range(3):
        var["W%d" % (l + 1)] = VdH[l].T @ lower[l] ** 2 + (dH[l] ** 2).T @ VA[l]
        var["b%d" % (l + 1)] = VdH[l].sum(0)
    var["W4"] = VdY.T @ A3 ** 2 + (dY ** 2).T @ VA[3]
    var["b4"] = VdY.sum(0)
    return {k: np.sqrt(v) for k, v in var.items()}


def test_gradients_match_oracle(S):
    """Every entry of every gradient tensor against the FP64 oracle on the same
    BF16 weights and FP32 biases, within K_SIGMA standard deviations of its own
    propagated BF16 rounding error (so one wrong row, column or bias entry
    cannot hide in a tensor norm)."""
    net, p, (shift, scale, mask, osh, osc) = _random_net(S, 3)
    rng = np.random.default_rng(4)
    M = 1000
    x = _raw_inputs(rng, M)
    t = np.stack([rng.normal(0.1, 0.2, M), rng.normal(-3.0, 1.5, M)], axis=1)
    try:
        g, L = net.gradients(torch.from_numpy(x.astype(np.float32)).cuda(),
                             torch.from_numpy(t.astype(np.float32)).cuda())
    finally:
        net.close()
    # the kernels multiply BF16 copies of the weights and add the FP32 biases
    Pm = omlp.unflatten(p)
    for name in ("W1", "W2", "W3", "W4"):
        Pm[name] = bf16_round(Pm[name].astype(np.float32))
    for name in ("b1", "b2", "b3", "b4"):
        Pm[name] = Pm[name].astype(np.float32).astype(np.float64)
    pm = omlp.flatten(Pm)
    xp = omlp.input_map(x.astype(np.float32).astype(np.float64), shift.astype(np.float32),
                        scale.astype(np.float32), mask)
    tp = (t.astype(np.float32) - osh) / osc
    L0, g0 = omlp.loss_and_grad(pm, xp, tp)
    assert abs(L - L0) <= 0.03 * L0
    G, G0 = omlp.unflatten(g.astype(np.float64)), omlp.unflatten(g0)
    sigma = _grad_error_sigma(pm, xp, tp, M)
    for name, _ in omlp.SHAPES:
        err, sg = np.abs(G[name] - G0[name]), sigma[name]
        if name == "W1":
            err, sg = err[:, :7], sg[:, :7]           # the padded input columns carry no gradient
        elif name in ("W4", "b4"):
            err, sg = err[:2], sg[:2]
        worst = float(np.max(err / (K_SIGMA * sg + 1e-12)))
        assert worst <= 1.0, (name, worst)
    # the bar has power: any entry of b2 off by 5 % of its own value, or one
    # entry of W3 off by 5 %, is rejected
    for name in ("b2", "W3"):
        ok = 0.05 * np.abs(G0[name]) > K_SIGMA * sigma[name]
        assert ok.mean() > 0.5, (name, ok.mean())



def test_adam_first_step(S):
    """t = 1: every live parameter moves by -lr sign(g) where the oracle's
    gradient is clearly non-zero (Adam's closed-form first step)."""
    net, p, (shift, scale, mask, osh, osc) = _random_net(S, 5)
    rng = np.random.default_rng(6)
    M, lr = 512, 1e-3
    x = _raw_inputs(rng, M)
    t = np.stack([rng.normal(0.1, 0.2, M), rng.normal(-3.0, 1.5, M)], axis=1)
    try:
        net.train_step(torch.from_numpy(x.astype(np.float32)).cuda(),
                       torch.from_numpy(t.astype(np.float32)).cuda(), lr)
        q = net.get_params().astype(np.float64)
    finally:
        net.close()
    pb = bf16_round(p)
    xp = omlp.input_map(x.astype(np.float32).astype(np.float64), shift.astype(np.float32),
                        scale.astype(np.float32), mask)
    _, g0 = omlp.loss_and_grad(pb, xp, (t.astype(np.float32) - osh) / osc)
    big = np.abs(g0) > 1e-3 * np.abs(g0).max()
    step = q - p.astype(np.float32).astype(np.float64)
    agree = np.abs(step[big] + lr * np.sign(g0[big])) <= 1e-6
    assert agree.mean() > 0.97, agree.mean()
    assert np.all(step[~big & (g0 == 0)] == 0)


def test_training_fits_a_smooth_function(S):
    rng = np.random.default_rng(7)
    N = 1 << 14
    x = _raw_inputs(rng, N)
    u = (x - x.min(0)) / (x.max(0) - x.min(0))
    t = np.stack([np.sin(3 * u[:, 3]) * np.cos(2 * u[:, 1]) + 0.5 * u[:, 0] * u[:, 6],
                  np.log10(x[:, 4]) + u[:, 2] ** 2], axis=1)
    net = S.Surrogate(8)
    try:
        lo = np.array([0.5, 2.0, 3.0, -0.3, -4.0, 0.1, 0.01])
        hi = np.array([1.5, 6.0, 7.0, 0.3, -1.0, 5.0, 0.5])
        net.set_maps((lo + hi) / 2, 2.0 / (hi - lo), 1 << 4, t.mean(0), t.std(0))
        X = torch.from_numpy(x.astype(np.float32)).cuda()
        T = torch.from_numpy(t.astype(np.float32)).cuda()
        hist = net.fit(X, T, steps=1500, batch=1024, lr=2e-3)
        y = net.forward(X).cpu().numpy()
    finally:
        net.close()
    assert hist[-50:].mean() < 0.05 * hist[:50].mean()
    rmse = np.sqrt(np.mean((y - t) ** 2, axis=0)) / t.std(0)
    assert np.all(rmse < 0.15), rmse


def _cosine_lr(lr, lr_final, k, steps):
    return lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * k / max(1, steps - 1)))


def test_fit_full_batch_matches_train_steps(S):
    """sde_mlp_fit with one minibatch per epoch (batch = N) against as many
    sde_mlp_train_step calls on the rows in their natural order, with the host's
    cosine learning rates.  The epoch's shuffled order must be a permutation of
    the rows (the loss before the first update is the full-data loss; a
    duplicated or missing row would move it by about 1/N), and the graph-replayed
    schedule and Adam corrections those of the host loop.  Only the summation
    order of the gradients' row reductions differs."""
    rng = np.random.default_rng(21)
    N, steps, lr, lr_final = 200, 6, 2e-3, 2e-4
    x = torch.from_numpy(_raw_inputs(rng, N).astype(np.float32)).cuda()
    t = torch.from_numpy(np.stack([rng.normal(0.1, 0.2, N), rng.normal(-3.0, 1.5, N)],
                                  axis=1).astype(np.float32)).cuda()
    nets = [_random_net(S, 22)[0] for _ in range(2)]
    try:
        hist = nets[0].fit(x, t, steps=steps, batch=N, lr=lr, lr_final=lr_final, seed=5)
        ref = torch.zeros(steps, dtype=torch.float32, device="cuda")
        for k in range(steps):
            nets[1].train_step(x, t, _cosine_lr(lr, lr_final, k, steps), loss_out=ref[k:k + 1])
        ref = ref.cpu().numpy()
        pa = nets[0].get_params().astype(np.float64)
        pb = nets[1].get_params().astype(np.float64)
    finally:
        for n in nets:
            n.close()
    np.testing.assert_allclose(hist[0], ref[0], rtol=1e-6)
    np.testing.assert_allclose(hist, ref, rtol=1e-5)
    assert hist[-1] < hist[0]
    # parameters: equal up to the reduction order (a weight whose gradient is
    # at rounding level may take Adam's sign step the other way)
    assert np.mean(np.abs(pa - pb) > 1e-5) < 0.01


def test_fit_rejects_bad_arguments(S):
    net = S.Surrogate(3)
    try:
        x = torch.zeros((16, 7), dtype=torch.float32, device="cuda")
        t = torch.zeros((16, 2), dtype=torch.float32, device="cuda")
        for kw in (dict(steps=0), dict(lr=0.0), dict(lr_final=-1.0)):
            with pytest.raises(Exception):
                net.fit(x, t, **dict(dict(steps=2, batch=8), **kw))
        rc = net._L.sde_mlp_fit(net._net, S._ptr(x), S._ptr(t), 16, 2, 17, 1e-3, 1e-4, 0.9, 0.999, 1e-8, 0, None)
        assert rc != 0                                           # batch > N
    finally:
        net.close()


def test_tcgen05_forward_matches_mma_path_and_oracle(S):
    """The fused tcgen05 forward (maps and layers 1-2; layers 3-4 and the
    output map; FP32 accumulators in tensor memory, two per CTA) against the
    layer-by-layer mma.sync kernels and the FP64 oracle, over a row count of
    521 tiles (several per CTA) ending in a ragged 128-row tile."""
    net, p, (shift, scale, mask, osh, osc) = _random_net(S, 9)
    rng = np.random.default_rng(10)
    M = 65536 + 1000 + 37
    x = _raw_inputs(rng, M)
    X = torch.from_numpy(x.astype(np.float32)).cuda()
    try:
        net.set_tensor_path(1)
        y_tc = net.forward(X)
        net.sync()
        net.set_tensor_path(0)
        y_mma = net.forward(X)
        net.sync()
        y_tc, y_mma = y_tc.cpu().numpy(), y_mma.cpu().numpy()
    finally:
        net.close()
    rms = np.sqrt(np.mean(((y_mma - osh) / osc) ** 2, axis=0))
    d = np.abs(y_tc - y_mma) / osc / rms
    assert np.isfinite(y_tc).all() and d.max() < 0.01, d.max()
    sel = np.concatenate([np.arange(300), np.arange(M - 300, M)])
    xp = omlp.input_map(x[sel].astype(np.float32).astype(np.float64), shift.astype(np.float32),
                        scale.astype(np.float32), mask)
    yp, _ = omlp.forward(bf16_round(p), xp)
    err = np.abs(y_tc[sel] - (yp * osc + osh)) / osc / np.sqrt(np.mean(yp ** 2, axis=0))
    assert err.max() < 0.03, err.max()


@pytest.mark.parametrize("M", [1, 127, 128, 129, 200, 152 * 128 + 5])
def test_tcgen05_forward_edge_sizes(S, M):
    """One row, a tile short of full, exactly one tile, one row past it, a
    tile whose last 32-row boxes of h2 lie past M (clipped and skipped tensor
    stores), and one more tile than SMs: the fused path agrees with the
    mma.sync path."""
    net, p, (shift, scale, mask, osh, osc) = _random_net(S, 12)
    x = _raw_inputs(np.random.default_rng(M), M)
    X = torch.from_numpy(x.astype(np.float32)).cuda()
    try:
        net.set_tensor_path(1)
        y_tc = net.forward(X)
        net.sync()
        net.set_tensor_path(0)
        y_mma = net.forward(X)
        net.sync()
        y_tc, y_mma = y_tc.cpu().numpy(), y_mma.cpu().numpy()
    finally:
        net.close()
    assert y_tc.shape == (M, 2) and np.isfinite(y_tc).all()
    d = np.abs(y_tc - y_mma) / osc
    assert d.max() < 0.02, d.max()

