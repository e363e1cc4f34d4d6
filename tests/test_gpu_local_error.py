"""GPU tests of Sec. 4's local-error indicator chi against the FP64 oracle,
and of the per-run step size chosen from it."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import engine
    engine.lib()
    return engine


@pytest.fixture(scope="module")
def W():
    from paper_1409_4923_gb300 import workloads
    return workloads


def _cases(W):
    pois = W.poisson_point()
    return {
        "inertial-deterministic": (0, dict(pois, Q=0.0, noise_flags=0), W.period_steps(4.9, 100)),
        "inertial-all-noises": (0, dict(pois, Fa=0.5, Fb=0.5, mua=2.0, mub=2.0, noise_flags=7),
                                W.period_steps(4.9, 100)),
        "inertial-dichot-drift": (0, dict(W.dichot_point(), noise_flags=1 | 4 | 32), W.period_steps(4.9, 200)),
        "overdamped-washboard": (1, dict(pois, V0=0.2, a=0.5, Q=0.05, Fa=0.3, Fb=0.6, mua=2.0, mub=1.0,
                                         noise_flags=7), 0.002),
    }


@pytest.mark.parametrize("case", ["inertial-deterministic", "inertial-all-noises", "inertial-dichot-drift",
                                  "overdamped-washboard"])
def test_chi_matches_oracle(E, W, orc, case):
    """Over one drive period (or 500 steps), where the FP32 paths still follow
    the FP64 ones: the RMS of chi within 1 %, its maximum within 5 %."""
    model, prm, dt = _cases(W)[case]
    n = int(round(2 * math.pi / 4.9 / dt)) if model == 0 else 500
    paths = 1024
    eng = E.Engine(model, E.make_params(**prm), seed=4)
    try:
        g = eng.local_error(paths, dt, n)
    finally:
        eng.close()
    d = dict(prm)
    d["noise"] = d.pop("noise_flags", 0)
    r = orc.local_error(model, orc.make_params(**d), 4, 0, paths, dt, n)
    for key in ("rms_x", "rms_v") if model == 0 else ("rms_x",):
        assert abs(g[key] / r[key] - 1) < 0.01, (key, g[key], r[key])
    for key in ("max_x", "max_v") if model == 0 else ("max_x",):
        assert abs(g[key] / r[key] - 1) < 0.05, (key, g[key], r[key])
    if model != 0:
        assert g["rms_v"] == 0.0


def test_suggested_step_meets_the_tolerance(E, W):
    from paper_1409_4923_gb300 import stepsize
    model, prm, _ = _cases(W)["inertial-deterministic"]
    eng = E.Engine(model, E.make_params(**prm), seed=1)
    try:
        tol = 2e-6
        s = stepsize.suggest_dt(eng, 0.02, tol, omega=4.9, paths=2048, component="rms_v")
        assert 2.5 < s["order"] < 3.5                     # local error O(dt^3) without noise
        period = 2 * math.pi / 4.9
        got = eng.local_error(2048, s["dt"], s["steps_per_period"])["rms_v"]
        assert s["steps_per_period"] * s["dt"] == pytest.approx(period)
        assert 0.5 * tol < got <= 1.05 * tol, (got, s)     # rounded up to whole steps per period
    finally:
        eng.close()
