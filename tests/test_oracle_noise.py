"""Pins of the oracle's noise increments (Algorithms 2-4) against their exact laws.

Three-point law: Eq. 25 (probabilities 1/6, 1/6, 2/3 of -c, +c, 0, c = G sqrt(3 dt)).
Poissonian noise: Eqs. 3-8 with the jump-adapted countdown of Algorithm 3;
  with an integer countdown drawn as floor(Exp(lambda)/dt) the event steps
  form an exact Bernoulli(p = 1 - exp(-lambda dt)) sequence, amplitudes are
  Exp(zeta) (Eq. 5), and between kicks the increment is -a dt (Eq. 6).
Dichotomous noise: Eqs. 13-17 with the countdown of Algorithm 4; per step the
  state -F_a is left with probability q_a = 1 - exp(-mu_a dt) and F_b with
  q_b = 1 - exp(-mu_b dt), so the stationary occupation of F_b is
  q_a / (q_a + q_b) and the correlation decays as (1 - q_a - q_b)^m, whose
  continuum limit is exp(-(mu_a + mu_b) t) (Eq. 15).
"""
import math

import numpy as np
import pytest
from scipy import stats as sst


def _seq(orc, kind, model, p, seed, paths, dt, n):
    return np.stack([orc.noise_sequence(kind, model, p, seed, i, dt, n) for i in range(paths)])


def test_three_point_law(orc):
    Q, dt = 0.5, 0.01
    p = orc.make_params(Q=Q, noise=orc.GAUSS)
    x = _seq(orc, 1, orc.OVERDAMPED_WASHBOARD, p, 3, 20, dt, 20000).ravel()
    G = math.sqrt(2 * Q)
    c = G * math.sqrt(3 * dt)
    vals = np.unique(x)
    assert len(vals) == 3
    np.testing.assert_allclose(vals, [-c, 0.0, c], rtol=0, atol=1e-15)
    counts = np.array([(x == -c).sum(), (x == c).sum(), (x == 0).sum()])
    exp = len(x) * np.array([1 / 6, 1 / 6, 2 / 3])
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 13.8, (counts, exp)                    # 2 dof, p = 0.001
    # moments of Eq. 25: E dxi^2 = G^2 dt, E dxi^4 = 3 G^4 dt^2
    m2, m4 = (x ** 2).mean(), (x ** 4).mean()
    se2 = (x ** 2).std() / math.sqrt(len(x))
    assert abs(m2 - G * G * dt) < 4 * se2
    assert abs(m4 - 3 * G ** 4 * dt ** 2) < 4 * (x ** 4).std() / math.sqrt(len(x))
    assert abs(x.mean()) < 4 * x.std() / math.sqrt(len(x))


def test_gaussian_increments(orc):
    Q, dt = 0.5, 0.01
    p = orc.make_params(Q=Q, noise=orc.GAUSS | orc.GAUSS_NORMAL)
    x = _seq(orc, 1, orc.OVERDAMPED_WASHBOARD, p, 5, 20, dt, 10000).ravel()
    s = math.sqrt(2 * Q * dt)
    assert abs(x.mean()) < 4 * s / math.sqrt(len(x))
    assert abs(x.var() / (s * s) - 1) < 4 * math.sqrt(2 / len(x))
    assert sst.kstest(x / s, "norm").pvalue > 1e-3
    lag1 = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(lag1) < 4 / math.sqrt(len(x))


@pytest.mark.parametrize("compensated", [False, True])
def test_poisson_increments(orc, compensated):
    lam, zeta, dt, n, M = 1.0, 0.1, 0.0128228, 4000, 300
    flags = orc.POISSON | (orc.POIS_COMPENSATED if compensated else 0)
    p = orc.make_params(**{"lambda": lam}, zeta=zeta, noise=flags)
    x = _seq(orc, 2, orc.OVERDAMPED_WASHBOARD, p, 11, M, dt, n)
    pe = 1 - math.exp(-lam * dt)
    aP = zeta * pe / dt if compensated else lam * zeta
    base = -aP * dt
    kick = x != base
    # counts over n steps ~ Binomial(n, pe)
    cnt = kick.sum(axis=1)
    mu, var = n * pe, n * pe * (1 - pe)
    assert abs(cnt.mean() - mu) < 4 * math.sqrt(var / M)
    assert abs(cnt.var(ddof=1) / var - 1) < 4 * math.sqrt(2 / M)
    # gaps between events are Geometric(pe) on {1, 2, ...}
    gaps = np.concatenate([np.diff(np.flatnonzero(r)) for r in kick])
    assert abs(gaps.mean() - 1 / pe) < 4 * math.sqrt((1 - pe) / pe ** 2 / len(gaps))
    # amplitudes ~ Exp(zeta)
    z = x[kick] - base
    assert sst.kstest(z, "expon", args=(0, zeta)).pvalue > 1e-3
    assert abs(z.mean() - zeta) < 4 * zeta / math.sqrt(len(z))
    # per-step mean of Delta eta: zeta pe - aP dt (zero when compensated)
    want = zeta * pe - aP * dt
    assert abs(x.mean() - want) < 4 * x.std() / math.sqrt(x.size)
    if compensated:
        assert abs(want) < 1e-15


def test_dichotomous_process(orc):
    Fa, Fb, mua, mub, dt, n, M = 1.0, 2.0, 1.0, 2.0, 0.01, 20000, 64
    p = orc.make_params(Fa=Fa, Fb=Fb, mua=mua, mub=mub, noise=orc.DICHOT)
    g = _seq(orc, 3, orc.OVERDAMPED_WASHBOARD, p, 21, M, dt, n)
    assert set(np.unique(g)) == {-Fa, Fb}
    qa, qb = 1 - math.exp(-mua * dt), 1 - math.exp(-mub * dt)
    occ = (g == Fb).mean(axis=1)
    want = qa / (qa + qb)
    assert abs(occ.mean() - want) < 4 * occ.std(ddof=1) / math.sqrt(M)
    # zero mean for Fa mu_b = Fb mu_a (Eq. 17)
    assert abs(g.mean()) < 4 * g.mean(axis=1).std(ddof=1) / math.sqrt(M)
    # correlation (1 - qa - qb)^m
    gc = g - g.mean()
    var = (gc * gc).mean()
    r = 1 - qa - qb
    for m in (10, 50, 150):
        per = (gc[:, :-m] * gc[:, m:]).mean(axis=1) / var
        assert abs(per.mean() - r ** m) < 4 * per.std(ddof=1) / math.sqrt(M) + 0.01, m
        # continuum limit of Eq. 15 differs from the discrete law by O(dt)
        assert abs(r ** m - math.exp(-(mua + mub) * m * dt)) < 0.01
    # mean sojourn in -F_a is 1 / qa steps
    sw = np.diff(np.flatnonzero(np.diff((g[0] == Fb).astype(np.int8)) != 0))
    assert len(sw) > 100


def test_three_point_steps_sharing_a_word_are_independent(orc):
    """Four consecutive steps share one Philox word (r, 6r, 36r, 216r mod 2^32):
    the 3 x 3 joint frequencies of each step and the next match the product
    law (1/6, 1/6, 2/3)^2, and so do steps 4 apart (different words)."""
    Q, dt = 0.5, 0.01
    p = orc.make_params(Q=Q, noise=orc.GAUSS)
    x = _seq(orc, 1, orc.OVERDAMPED_WASHBOARD, p, 13, 40, dt, 16000)
    c = math.sqrt(2 * Q) * math.sqrt(3 * dt)
    cls = np.where(x < 0, 0, np.where(x > 0, 1, 2))
    probs = np.array([1 / 6, 1 / 6, 2 / 3])
    for lag in (1, 2, 3, 4):
        for k in range(4):                       # position within the word
            a = cls[:, k:-lag:4] if lag < 4 else cls[:, k::4][:, :-1]
            b = cls[:, k + lag::4][:, :a.shape[1]]
            a, b = a.ravel()[:b.size], b.ravel()
            obs = np.zeros((3, 3))
            np.add.at(obs, (a, b), 1)
            exp = np.outer(probs, probs) * a.size
            chi2 = ((obs - exp) ** 2 / exp).sum()
            assert chi2 < 26.1, (lag, k, chi2)   # 8 dof, p = 0.001
    assert abs(np.abs(x[x != 0]).mean() - c) < 1e-15


def test_three_point_four_steps_of_one_word_jointly_independent(orc):
    """All 81 joint outcomes of the four steps that share one Philox word
    (uniforms r, 6r, 36r, 216r mod 2^32; Algorithm 2 draws a fresh uniform per
    step) against the product law of Eq. 25's three-point distribution,
    (1/6, 1/6, 2/3)^4: a chi-square test with 80 degrees of freedom, which sees
    any dependence among the four digits of one word, not only pairwise lags."""
    Q, dt = 0.5, 0.01
    p = orc.make_params(Q=Q, noise=orc.GAUSS)
    x = _seq(orc, 1, orc.OVERDAMPED_WASHBOARD, p, 17, 64, dt, 16000)
    cls = np.where(x < 0, 0, np.where(x > 0, 1, 2))
    words = cls.reshape(cls.shape[0], -1, 4).reshape(-1, 4)        # steps 4i .. 4i + 3
    cell = ((words[:, 0] * 3 + words[:, 1]) * 3 + words[:, 2]) * 3 + words[:, 3]
    obs = np.bincount(cell, minlength=81).astype(np.float64)
    probs = np.array([1 / 6, 1 / 6, 2 / 3])
    exp = np.einsum("i,j,k,l->ijkl", probs, probs, probs, probs).ravel() * len(cell)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < sst.chi2.ppf(0.999, 80), chi2
    # and the test has power: 10 % of the words with their last digit copied
    # from the first (a dependence a pairwise lag-3 test would also see, here
    # one of 81 cells) is rejected
    bad = words.copy()
    sel = np.arange(len(bad)) % 10 == 0
    bad[sel, 3] = bad[sel, 0]
    cb = ((bad[:, 0] * 3 + bad[:, 1]) * 3 + bad[:, 2]) * 3 + bad[:, 3]
    ob = np.bincount(cb, minlength=81).astype(np.float64)
    assert ((ob - exp) ** 2 / exp).sum() > sst.chi2.ppf(0.999, 80)
