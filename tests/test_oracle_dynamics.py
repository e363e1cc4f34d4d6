"""Pins of the oracle's integrator (Algorithm 1 with Algorithms 2-4) and of the
Eq. 31 estimator against closed forms and exact laws of the discrete scheme.

Every tolerance is a few standard errors of the Monte Carlo estimate plus, where
the comparison is with a continuum result, an allowance for the scheme's
discretisation error (stated at each check).
"""
import math
import os

import numpy as np
import pytest

import closed_forms as cf


def _paper_settings():
    """The validation settings the paper states for Models I and II (Sec. 6 and
    the Fig. 3 caption), from tests/golden/paper_validation_settings.txt:
    {model: {key: value or list of values}}."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_validation_settings.txt")
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, *items = line.split()
            d = {}
            for item in items:
                k, v = item.split("=")
                vals = [float(x) for x in v.split(",")]
                d[k] = vals if len(vals) > 1 else vals[0]
            out[name] = d
    return out


PAPER = _paper_settings()


def test_paper_settings_fixture():
    assert PAPER["model_I"]["a"] == [1.5, 2.5] and PAPER["model_I"]["spp"] == 400
    assert PAPER["model_II"]["Fa"] == 3 and PAPER["model_II"]["Fb"] == [1.1, 1.6]
    assert PAPER["model_II"]["spp"] == 200
    assert PAPER["model_I"]["DG"] == 0 and PAPER["model_II"]["DG"] == 0
    assert PAPER["model_I"]["transient_fraction"] == PAPER["model_II"]["transient_fraction"] == 0.1


def _var_se(x):
    """Sample variance and its standard error (from the fourth central moment)."""
    x = np.asarray(x, dtype=np.float64)
    c = x - x.mean()
    v = (c * c).mean()
    m4 = (c ** 4).mean()
    return v, math.sqrt(max(m4 - v * v, 0.0) / len(x))


# ---------------------------------------------------------------- free particle

@pytest.mark.parametrize("normal", [False, True])
def test_free_diffusion(orc, normal):
    """Overdamped, no force: <x^2> = 2 D t exactly for the discrete scheme."""
    Q, dt, n, M = 0.5, 0.01, 1000, 20000
    flags = orc.GAUSS | (orc.GAUSS_NORMAL if normal else 0)
    p = orc.make_params(V0=0.0, Q=Q, noise=flags)
    r = orc.run_paths(orc.OVERDAMPED_WASHBOARD, p, 1, 0, M, dt, 0, n)
    x = r["X_f"]
    v, se = _var_se(x)
    assert abs(v - 2 * Q * n * dt) < 4 * se
    assert abs(x.mean()) < 4 * math.sqrt(v / M)
    np.testing.assert_array_equal(r["X_i"], 0.0)


def test_ornstein_uhlenbeck_mean_order_two(orc):
    """x' = -k x, Algorithm 1 gives x_{n+1} = alpha x_n with
    alpha = 1 - h + h^2/2 - h^3/4 (h = k dt): exact recursion, weak order 2."""
    k, T = 1.0, 2.0
    errs = []
    for h in (0.1, 0.05, 0.025, 0.0125):
        dt = h / k
        n = int(round(T / dt))
        p = orc.make_params(V0=k, x0_lo=1.0, x0_hi=1.0)
        r = orc.run_paths(orc.OVERDAMPED_LINEAR, p, 0, 0, 1, dt, 0, n)
        alpha = 1 - h + h * h / 2 - h ** 3 / 4
        assert abs(r["X_f"][0] - alpha ** n) < 1e-13
        errs.append(abs(r["X_f"][0] - math.exp(-k * T)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(1.9 < s < 2.2 for s in slopes) and abs(slopes[-1] - 2) < 0.05, slopes


@pytest.mark.parametrize("normal", [False, True])
def test_ornstein_uhlenbeck_variance(orc, normal):
    """Var x_{n+1} = alpha^2 Var x_n + beta^2 2 D dt, beta = 1 - h/2 + h^2/4."""
    k, D, dt, n, M = 1.0, 0.5, 0.1, 30, 40000
    h = k * dt
    alpha = 1 - h + h * h / 2 - h ** 3 / 4
    beta = 1 - h / 2 + h * h / 4
    var = 0.0
    for _ in range(n):
        var = alpha * alpha * var + beta * beta * 2 * D * dt
    flags = orc.GAUSS | (orc.GAUSS_NORMAL if normal else 0)
    p = orc.make_params(V0=k, Q=D, x0_lo=1.0, x0_hi=1.0, noise=flags)
    r = orc.run_paths(orc.OVERDAMPED_LINEAR, p, 2, 0, M, dt, 0, n)
    v, se = _var_se(r["X_f"])
    assert abs(v - var) < 4 * se
    assert abs(r["X_f"].mean() - alpha ** n) < 4 * math.sqrt(var / M)
    # and the recursion is within O(h^2) of the continuum D/k (1 - e^{-2kt})
    assert abs(var - D / k * (1 - math.exp(-2 * k * n * dt))) < 0.01


def test_inertial_free_covariance(orc):
    """x' = v, v' = -g v + sqrt(2 g Q) xi.  Algorithm 1 on y = (x, v) gives the
    exact linear recursion y' = M y + b dxi with
      M = [[1, h (1 - gh/2 + g^2 h^2/4)], [0, 1 - gh + g^2 h^2/2 - g^3 h^3/4]],
      b = [h/2 (1 - gh/2), 1 - gh/2 + g^2 h^2/4]."""
    g, Q, dt, n, M_ = 0.9, 0.5, 0.05, 200, 20000
    h = dt
    Mm = np.array([[1.0, h * (1 - g * h / 2 + g * g * h * h / 4)],
                   [0.0, 1 - g * h + g * g * h * h / 2 - g ** 3 * h ** 3 / 4]])
    b = np.array([h / 2 * (1 - g * h / 2), 1 - g * h / 2 + g * g * h * h / 4])
    C = np.zeros((2, 2))
    for _ in range(n):
        C = Mm @ C @ Mm.T + np.outer(b, b) * 2 * g * Q * dt
    p = orc.make_params(gamma=g, Q=Q, V0=0.0, noise=orc.GAUSS)
    r = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 4, 0, M_, dt, 0, n)
    x, v = r["X_f"], r["v_f"]
    vx, sex = _var_se(x)
    vv, sev = _var_se(v)
    assert abs(vx - C[0, 0]) < 4 * sex
    assert abs(vv - C[1, 1]) < 4 * sev
    cxv = ((x - x.mean()) * (v - v.mean())).mean()
    se_c = ((x - x.mean()) * (v - v.mean())).std() / math.sqrt(M_)
    assert abs(cxv - C[0, 1]) < 4 * se_c
    # the recursion tends to the continuum covariance at second order
    xx, xv, vvc = cf.inertial_free_variance(g, Q, n * dt)
    assert abs(C[1, 1] - vvc) < 0.01 * vvc and abs(C[0, 0] - xx) < 0.01 * xx


def test_inertial_driven_linear_deterministic(orc):
    """Noise-free v' = -g v + a cos(w t) + F: second-order convergence of the
    trapezoidal predictor-corrector to the exact solution (checks the drive's
    sign, frequency, phase at t_{n+1} and the bias)."""
    g, a, w, F, v0, T = 0.9, 4.2, 4.9, 0.1, 1.0, 5.0
    ev, ex = [], []
    for dt in (0.02, 0.01, 0.005):
        n = int(round(T / dt))
        p = orc.make_params(gamma=g, a=a, omega=w, F=F, V0=0.0, v0_lo=v0, v0_hi=v0)
        r = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 0, 0, 1, dt, 0, n)
        ev.append(abs(r["v_f"][0] - cf.driven_linear_velocity(g, a, w, F, v0, T)))
        ex.append(abs(r["X_f"][0] - cf.driven_linear_position(g, a, w, F, v0, T)))
    assert ev[-1] < 1e-4 and ex[-1] < 1e-4
    for e in (ev, ex):
        s = [math.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(1.8 < x < 2.2 for x in s), (ev, ex)


def test_inertial_driven_washboard_deterministic(orc):
    """The bench's nonlinear model with the noise off, x'' = -g x' - 2 pi V0
    cos(2 pi x) + a cos(w t) + F (washboard V0 sin(2 pi x), drive and bias),
    over one drive period from fixed (x0, v0): the scheme converges at second
    order to SciPy's DOP853 solution at 1e-13 tolerances.  This pins the
    washboard force's sign, factor and argument together with the drive and the
    damping of the model the engine is timed on (the linear tests above cover
    the drive alone).  One period keeps the chaotic growth of trajectory
    differences out of the comparison."""
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    g, a, w, F, V0, x0, v0 = 0.9, 4.2, 4.9, 0.1, 1.0, 0.3, 0.7
    T = 2 * math.pi / w

    def rhs(t, y):
        return [y[1], -g * y[1] - 2 * math.pi * V0 * math.cos(2 * math.pi * y[0]) + a * math.cos(w * t) + F]

    ref = solve_ivp(rhs, (0.0, T), [x0, v0], method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    ex, ev = [], []
    for n in (200, 400, 800):
        p = orc.make_params(gamma=g, a=a, omega=w, F=F, V0=V0, x0_lo=x0, x0_hi=x0, v0_lo=v0, v0_hi=v0)
        r = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 0, 0, 1, T / n, 0, n)
        ex.append(abs(r["X_f"][0] - ref[0]))
        ev.append(abs(r["v_f"][0] - ref[1]))
    assert ex[-1] < 5e-6 and ev[-1] < 1e-5, (ex, ev)
    sx = [math.log2(ex[i] / ex[i + 1]) for i in range(2)]
    sv = [math.log2(ev[i] / ev[i + 1]) for i in range(2)]
    assert all(1.9 < x < 2.1 for x in sx), sx
    assert all(1.9 < x < 2.7 for x in sv), sv          # v approaches order 2 from above


def test_overdamped_driven_deterministic(orc):
    """Noise-free x' = a cos(w t) + F: x(T) = F T + (a / w) sin(w T) to O(dt^2)."""
    a, w, F, T = 1.3, 2.0, 0.7, 3.0
    errs = []
    for dt in (0.01, 0.005):
        n = int(round(T / dt))
        p = orc.make_params(a=a, omega=w, F=F, V0=0.0)
        r = orc.run_paths(orc.OVERDAMPED_WASHBOARD, p, 0, 0, 1, dt, 0, n)
        errs.append(abs(r["X_f"][0] - (F * T + a / w * math.sin(w * T))))
    assert errs[-1] < 1e-5 and 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("model", ["inertial", "linear"])
def test_dichotomous_force_as_drift_is_second_order(orc, model):
    """Frozen dichotomous force (rates so small that no flip happens) and no
    other force: v' = -g v + Gamma (inertial) or x' = -k x + Gamma (linear
    force) have the closed form y(T) = Gamma/g + (y0 - Gamma/g) e^{-g T}.
    As a drift term (DICHOT_IN_DRIFT) Gamma is integrated by the
    predictor-corrector, whose error falls 4x per halving of dt; as Algorithm
    1's corrector increment it is a first-order splitting (2x).  A term
    dropped from one of the three drift evaluations, or Gamma counted twice,
    breaks one of the two rates."""
    g, b, y0, T = 0.9, 0.5, 1.0, 4.0
    for flags, lo, hi in ((orc.DICHOT | orc.DICHOT_IN_DRIFT, 3.9, 4.2), (orc.DICHOT, 1.95, 2.05)):
        errs = []
        for dt in (0.04, 0.02, 0.01):
            n = int(round(T / dt))
            if model == "inertial":
                p = orc.make_params(gamma=g, V0=0.0, Fa=b, Fb=b, mua=1e-9, mub=1e-9, v0_lo=y0,
                                    v0_hi=y0, noise=flags)
                r = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 0, 0, 16, dt, 0, n)
                y = r["v_f"]
            else:
                p = orc.make_params(V0=g, Fa=b, Fb=b, mua=1e-9, mub=1e-9, x0_lo=y0, x0_hi=y0,
                                    noise=flags)
                r = orc.run_paths(orc.OVERDAMPED_LINEAR, p, 0, 0, 16, dt, 0, n)
                y = r["X_f"]
            assert (r["jD"] == 0).all() and set(r["d"]) == {0, 1}     # frozen, both states seen
            G = np.where(r["d"] == 1, b, -b)
            errs.append(np.abs(y - (G / g + (y0 - G / g) * math.exp(-g * T))).max())
        rates = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(lo < q < hi for q in rates), (flags, errs)


def test_local_error_chi_closed_form(orc):
    """Sec. 4's chi = predictor - corrector.  For x' = -k x, Algorithm 1 gives
    Euler x(1 - h), predictor x(1 - h + h^2/2), corrector
    x(1 - h + h^2/2 - h^3/4) with h = k dt, so chi_n = x_n h^3 / 4 exactly, on
    x_n = x0 alpha^n with alpha the corrector's factor."""
    k, x0, n = 0.9, 1.0, 40
    for dt in (0.1, 0.05, 0.025):
        h = k * dt
        alpha = 1.0 - h + h * h / 2.0 - h ** 3 / 4.0
        chi = x0 * alpha ** np.arange(n) * h ** 3 / 4.0
        r = orc.local_error(orc.OVERDAMPED_LINEAR, orc.make_params(V0=k, x0_lo=x0, x0_hi=x0), 0, 0, 4, dt, n)
        assert abs(r["rms_x"] / math.sqrt(np.mean(chi ** 2)) - 1.0) < 1e-9
        assert abs(r["max_x"] / chi[0] - 1.0) < 1e-9
        assert r["rms_v"] == 0.0


@pytest.mark.parametrize("model", [0, 1])
def test_local_error_scales_as_dt_cubed(orc, model):
    """Noise-free washboards: chi is the local error of a second-order scheme,
    O(dt^3): halving dt divides it by about 8 (inertial: both components)."""
    kw = (dict(gamma=0.9, a=4.2, omega=4.9, F=0.1, v0_lo=-2.0, v0_hi=2.0) if model == 0 else
          dict(V0=0.2, a=0.5, omega=4.9, F=0.1))
    rs = [orc.local_error(model, orc.make_params(x0_hi=1.0, **kw), 0, 0, 64, dt, int(round(1.0 / dt)))
          for dt in (0.02, 0.01, 0.005)]
    for key in (("rms_x", "rms_v") if model == 0 else ("rms_x",)):
        for a, b in zip(rs[:-1], rs[1:]):
            assert 7.0 < a[key] / b[key] < 9.0, (key, a[key] / b[key])


def test_local_error_excludes_jumps(orc):
    """The jump increments are exact and enter only the corrector: a force-free
    overdamped particle under Poisson and dichotomous noise has chi = 0."""
    p = orc.make_params(V0=0.0, zeta=0.3, Fa=0.5, Fb=0.5, mua=2.0, mub=2.0, noise=orc.POISSON | orc.DICHOT,
                        **{"lambda": 3.0})
    r = orc.local_error(orc.OVERDAMPED_WASHBOARD, p, 0, 0, 16, 0.01, 500)
    assert r["max_x"] < 1e-15


@pytest.mark.parametrize("compensated", [False, True])
def test_poisson_free_particle(orc, compensated):
    """Overdamped, no force, Poisson only: x_n - x_0 is a sum of n i.i.d. increments
    (Bernoulli(p) kicks of Exp(zeta) size minus a dt): mean n (zeta p - a dt),
    variance n (2 p zeta^2 - p^2 zeta^2)."""
    lam, zeta, dt, n, M = 1.0, 0.1, 0.0128228, 1000, 20000
    flags = orc.POISSON | (orc.POIS_COMPENSATED if compensated else 0)
    p = orc.make_params(**{"lambda": lam}, zeta=zeta, V0=0.0, noise=flags)
    r = orc.run_paths(orc.OVERDAMPED_WASHBOARD, p, 7, 0, M, dt, 0, n)
    pe = 1 - math.exp(-lam * dt)
    aP = zeta * pe / dt if compensated else lam * zeta
    mean = n * (zeta * pe - aP * dt)
    var = n * (2 * pe * zeta ** 2 - pe * pe * zeta ** 2)
    x = r["X_f"]
    assert abs(x.mean() - mean) < 4 * math.sqrt(var / M)
    v, se = _var_se(x)
    assert abs(v - var) < 4 * se


# ---------------------------------------------------------------- potentials

@pytest.mark.parametrize("V0,F,D", [(1.0, 5.0, 1.0), (1 / (2 * math.pi), 0.5, 0.1)])
def test_stratonovich_tilted_washboard(orc, V0, F, D):
    """Overdamped tilted washboard: <v> of Eq. 31 vs Stratonovich's closed form,
    within 4 SE plus an O(dt^2) allowance of 0.3 % of F."""
    dt, n, M = 0.002, 20000, 2048
    want = cf.stratonovich_velocity(V0, F, D)
    p = orc.make_params(V0=V0, F=F, Q=D, x0_hi=1.0, noise=orc.GAUSS)
    r = orc.run_paths(orc.OVERDAMPED_WASHBOARD, p, 0, 0, M, dt, 2000, n)
    s = orc.stats(r, n)
    assert abs(s["mean_v"] - want) < 4 * s["stderr_v"] + 0.003 * F


@pytest.mark.slow
@pytest.mark.parametrize("a,DP", list(zip(PAPER["model_I"]["a"], (1.0, 2.0))))
def test_model_I_eq21a(orc, a, DP):
    """Model I (Eq. 1), D_G = 0, L = 2: <v> = 2 J_I (Eqs. 21a-23), settings of the
    paper's validation (spp = 400, dt = (1/lambda)/400, 10 % transient dropped).
    The compensated bias makes the kick process exactly zero-mean; the residual
    discretisation allowance is 0.003."""
    cfg = PAPER["model_I"]
    lam, zeta = a * a / DP, DP / a
    dt = (1 / lam) / cfg["spp"]
    n = int(200 / lam / dt)                       # 200 mean kick intervals (the paper: 1000)
    n_tr = int(round(n * cfg["transient_fraction"]))
    p = orc.make_params(**{"lambda": lam}, zeta=zeta, x0_lo=-1.0, x0_hi=1.0,
                        noise=orc.POISSON | orc.POIS_COMPENSATED)
    r = orc.run_paths(orc.OVERDAMPED_PWL, p, 0, 0, 2048, dt, n_tr, n - n_tr)
    s = orc.stats(r, n - n_tr)
    want = cf.eq21a_velocity(a, DP)
    assert abs(s["mean_v"] - want) < 4 * s["stderr_v"] + 0.003, (s, want)


@pytest.mark.slow
@pytest.mark.parametrize("Fb,tau", list(zip(PAPER["model_II"]["Fb"], (1.0, 0.5))))
def test_model_II_eq21b_corrected_sign(orc, Fb, tau):
    """Model II (Eq. 12), D_G = 0, F_a = 3 (the paper's validation values), zero
    mean (F_a mu_b = F_b mu_a).  Matches Eq. 21b with (beta_- - beta_+) and
    rejects the printed sign."""
    cfg = PAPER["model_II"]
    Fa = cfg["Fa"]
    mua, mub = Fa / (tau * (Fa + Fb)), Fb / (tau * (Fa + Fb))
    ref = min(1 / mua, 1 / mub)
    dt = ref / cfg["spp"]
    n = int(400 * ref / dt)                       # 400 x min(tau_a, tau_b) (the paper: 1000)
    n_tr = int(round(n * cfg["transient_fraction"]))
    p = orc.make_params(Fa=Fa, Fb=Fb, mua=mua, mub=mub, x0_lo=-1.0, x0_hi=1.0,
                        noise=orc.DICHOT)
    r = orc.run_paths(orc.OVERDAMPED_PWL, p, 0, 0, 2048, dt, n_tr, n - n_tr)
    s = orc.stats(r, n - n_tr)
    want = cf.eq21b_velocity(Fa, Fb, tau)
    printed = cf.eq21b_velocity(Fa, Fb, tau, printed_sign=True)
    assert abs(s["mean_v"] - want) < 4 * s["stderr_v"] + 0.005, (s, want)
    assert abs(s["mean_v"] - printed) > 20 * s["stderr_v"]


def test_eq21b_adiabatic_limit():
    """tau -> oo: <v> -> P_b v(F_b) + P_a v(-F_a) with the sliding velocities."""
    Fa, Fb = 3.0, 1.1
    Pb, Pa = Fa / (Fa + Fb), Fb / (Fa + Fb)
    lim = Pb * cf.pwl_sliding_velocity(Fb) + Pa * cf.pwl_sliding_velocity(-Fa)
    assert abs(cf.eq21b_velocity(Fa, Fb, 1e5) - lim) < 1e-3
    assert abs(cf.eq21b_velocity(Fa, Fb, 1e5, printed_sign=True) + lim) < 1e-3


def test_equipartition_inertial_washboard(orc):
    """Undriven, untilted inertial washboard at thermal equilibrium: <v> = 0 and
    <v^2> = Q for any potential (Maxwell velocity law), to O(dt^2)."""
    g, Q, dt, ntr, n, M = 0.9, 0.5, 0.01, 2000, 20000, 512
    p = orc.make_params(gamma=g, Q=Q, x0_hi=1.0, noise=orc.GAUSS)
    r = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 8, 0, M, dt, ntr, n)
    per_v2 = r["sum_v2"] / n
    assert abs(per_v2.mean() - Q) < 4 * per_v2.std(ddof=1) / math.sqrt(M) + 0.002
    s = orc.stats(r, n)
    assert abs(s["mean_v"]) < 4 * s["stderr_v"]
    assert abs(s["tmean_v"]) < 4 * (r["sum_v"] / n).std(ddof=1) / math.sqrt(M)


# ---------------------------------------------------------------- estimator

def test_window_and_restart_consistency(orc):
    """Eq. 31 window: splitting the same steps into transient + average changes
    neither the trajectory nor the final state; vbar = (X_f - X_i) / (n_avg dt)."""
    p = orc.make_params(gamma=0.9, a=4.2, omega=4.9, F=0.1, Q=0.001, **{"lambda": 1.0},
                        zeta=0.1, x0_hi=1.0, v0_lo=-2.0, v0_hi=2.0,
                        noise=orc.GAUSS | orc.POISSON)
    dt = (2 * math.pi / 4.9) / 100
    a = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 0, 0, 16, dt, 0, 600)
    b = orc.run_paths(orc.INERTIAL_WASHBOARD, p, 0, 0, 16, dt, 200, 400)
    np.testing.assert_array_equal(a["X_f"], b["X_f"])
    np.testing.assert_array_equal(a["v_f"], b["v_f"])
    np.testing.assert_array_equal(a["jP"], b["jP"])
    np.testing.assert_allclose(b["vbar"], (b["X_f"] - b["X_i"]) / (400 * dt), rtol=1e-14)


def test_stats_two_pass(orc):
    rng = np.random.default_rng(0)
    rec = np.zeros(1000, dtype=orc.PATH_DTYPE)
    rec["vbar"] = 0.3 + 1e-3 * rng.standard_normal(1000)
    rec["sum_v"] = rng.standard_normal(1000)
    rec["sum_v2"] = rng.random(1000)
    s = orc.stats(rec, 10)
    assert s["n"] == 1000
    assert abs(s["mean_v"] - rec["vbar"].mean()) < 1e-15
    assert abs(s["var_v"] / rec["vbar"].var(ddof=1) - 1) < 1e-12
    assert abs(s["stderr_v"] - math.sqrt(rec["vbar"].var(ddof=1) / 1000)) < 1e-15
    tm = rec["sum_v"].sum() / 10000
    assert abs(s["tmean_v"] - tm) < 1e-15
    assert abs(s["tvar_v"] - (rec["sum_v2"].sum() / 10000 - tm * tm)) < 1e-14
