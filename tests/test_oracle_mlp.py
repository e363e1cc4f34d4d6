"""Pins of the FP64 surrogate-network oracle: hand-written backward pass against
central finite differences, Adam's first step against its closed form."""
import numpy as np

from oracle import mlp


def _setup(seed=0, M=12):
    rng = np.random.default_rng(seed)
    p = np.zeros(mlp.NPARAMS)
    P = mlp.unflatten(p)
    for name, shape in mlp.SHAPES:
        P[name] = rng.standard_normal(shape) * (0.3 if name.startswith("W") else 0.1)
    P["W1"][:, mlp.IN:] = 0.0
    P["W4"][mlp.OUT:, :] = 0.0
    P["b4"][mlp.OUT:] = 0.0
    p = mlp.flatten(P)
    x = rng.uniform(0.5, 2.0, size=(M, mlp.IN))
    xp = mlp.input_map(x, np.full(7, 1.0), np.full(7, 0.8), 0b0010000)
    tp = rng.standard_normal((M, mlp.OUT))
    return p, xp, tp


def test_gradients_match_central_differences():
    p, xp, tp = _setup()
    L, g = mlp.loss_and_grad(p, xp, tp)
    assert abs(L - mlp.loss(p, xp, tp)) < 1e-15
    rng = np.random.default_rng(1)
    live = [i for i in range(mlp.NPARAMS)]
    idx = rng.choice(live, size=400, replace=False)
    P = mlp.unflatten(np.arange(mlp.NPARAMS, dtype=np.float64))
    # every tensor is represented
    idx = np.concatenate([idx, [int(P[n].ravel()[0]) for n, _ in mlp.SHAPES]])
    for i in idx:
        h = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(pp, xp, tp) - mlp.loss(pm, xp, tp)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_padding_gets_no_gradient():
    p, xp, tp = _setup(2)
    _, g = mlp.loss_and_grad(p, xp, tp)
    G = mlp.unflatten(g)
    assert np.all(G["W1"][:, mlp.IN:] == 0.0)
    assert np.all(G["W4"][mlp.OUT:, :] == 0.0) and np.all(G["b4"][mlp.OUT:] == 0.0)


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected ratio is g / |g|: every parameter moves by
    -lr sign(g) (up to eps)."""
    rng = np.random.default_rng(3)
    p = rng.standard_normal(1000)
    g = rng.standard_normal(1000)
    z = np.zeros(1000)
    q, m1, m2 = mlp.adam_step(p, g, z, z, 1, 1e-3, eps=1e-12)
    np.testing.assert_allclose(q - p, -1e-3 * np.sign(g), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 0.001 * g * g)


def test_silu_derivative():
    x = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(x), (mlp.silu(x + h) - mlp.silu(x - h)) / (2 * h), rtol=1e-7,
                               atol=1e-9)
