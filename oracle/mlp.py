"""FP64 numpy oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

Plain float64 forward pass, hand-written backward pass and Adam for the
network 7 -> 256 -> 256 -> 256 -> 2 with SiLU hidden activations, on the same
flat, padded parameter vector the engine exposes (an interface both sides
must share): W1[256][16], b1[256], W2[256][256], b2[256], W3[256][256],
b3[256], W4[8][256], b4[8].  Only tests/ and bench.py may use it.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss
(relative 1e-6) and the closed-form first Adam step.
"""
import numpy as np

IN, IN_PAD, H, OUT, OUT_PAD = 7, 16, 256, 2, 8
SHAPES = [("W1", (H, IN_PAD)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
          ("b3", (H,)), ("W4", (OUT_PAD, H)), ("b4", (OUT_PAD,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(p):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def input_map(x, shift, scale, log_mask):
    """x' = (g(x) - shift) * scale, g = log10 on the masked features, padded to 16."""
    x = np.asarray(x, dtype=np.float64).copy()
    for c in range(IN):
        if log_mask >> c & 1:
            x[:, c] = np.log10(x[:, c])
    xp = np.zeros((x.shape[0], IN_PAD))
    xp[:, :IN] = (x - np.asarray(shift, dtype=np.float64)) * np.asarray(scale, dtype=np.float64)
    return xp


def forward(p, xp):
    """Standardised outputs y' [M][2] and the intermediates of the backward pass."""
    P = unflatten(p)
    H1 = xp @ P["W1"].T + P["b1"]
    A1 = silu(H1)
    H2 = A1 @ P["W2"].T + P["b2"]
    A2 = silu(H2)
    H3 = A2 @ P["W3"].T + P["b3"]
    A3 = silu(H3)
    Y = A3 @ P["W4"].T + P["b4"]
    return Y[:, :OUT], (xp, H1, A1, H2, A2, H3, A3, Y)


def loss_and_grad(p, xp, tp):
    """L = 1/(2M) sum (y' - t')^2 and dL/dp (flat, padded layout)."""
    P = unflatten(p)
    y, (X, H1, A1, H2, A2, H3, A3, Y) = forward(p, xp)
    M = X.shape[0]
    R = y - tp
    L = 0.5 * np.sum(R * R) / M
    dY = np.zeros_like(Y)
    dY[:, :OUT] = R / M
    g = {"W4": dY.T @ A3, "b4": dY.sum(0)}
    dH3 = (dY @ P["W4"]) * dsilu(H3)
    g["W3"], g["b3"] = dH3.T @ A2, dH3.sum(0)
    dH2 = (dH3 @ P["W3"]) * dsilu(H2)
    g["W2"], g["b2"] = dH2.T @ A1, dH2.sum(0)
    dH1 = (dH2 @ P["W2"]) * dsilu(H1)
    g["W1"], g["b1"] = dH1.T @ X, dH1.sum(0)
    return L, flatten(g)


def loss(p, xp, tp):
    y, _ = forward(p, xp)
    R = y - tp
    return 0.5 * np.sum(R * R) / xp.shape[0]


def adam_step(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) at step t >= 1; returns new (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
