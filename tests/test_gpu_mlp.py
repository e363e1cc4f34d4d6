"""GPU tests of the surrogate network's kernels against the FP64 oracle.

Bars: GEMM entries within 1e-5 of the float64 product of the same BF16
operands, relative to sum |a||b| (FP32 accumulation); forward outputs within
3 % of the RMS of the standardised output and gradients within 5 % (norm-wise,
per tensor) of
the FP64 oracle evaluated on the same BF16-rounded weights (the kernels round
every activation to BF16, 2^-9 relative, through four layers).
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


def test_gradients_match_oracle(S):
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
    pb = bf16_round(p)
    xp = omlp.input_map(x.astype(np.float32).astype(np.float64), shift.astype(np.float32),
                        scale.astype(np.float32), mask)
    tp = (t.astype(np.float32) - osh) / osc
    L0, g0 = omlp.loss_and_grad(pb, xp, tp)
    assert abs(L - L0) <= 0.03 * L0
    G, G0 = omlp.unflatten(g.astype(np.float64)), omlp.unflatten(g0)
    for name, _ in omlp.SHAPES:
        rel = np.linalg.norm(G[name] - G0[name]) / (np.linalg.norm(G0[name]) + 1e-30)
        assert rel < 0.05, (name, rel)
    assert np.all(G["W1"][:, 7:] == 0) and np.all(G["W4"][2:] == 0)


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


@pytest.mark.parametrize("M", [1, 127, 128, 129, 152 * 128 + 5])
def test_tcgen05_forward_edge_sizes(S, M):
    """One row, a tile short of full, exactly one tile, one row past it, and
    one more tile than SMs: the fused path agrees with the mma.sync path."""
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

