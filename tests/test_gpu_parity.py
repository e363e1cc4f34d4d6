"""GPU parity: the CUDA engine (through the C ABI) against the FP64 oracle.

Bars (derivation in the design notes):
  - integers (Philox words, event indices, counts): bit-exact;
  - per path over short horizons (<= 64 steps): |dX| <= 2e-5 and |dv| <= 2e-4
    (FP32 state rounding and SFU cosine error, amplified by the local
    instability of the driven washboard), on every path; piecewise-linear
    paths whose force was evaluated within 1e-5 of a kink are excluded
    because FP32 and FP64 may take the two sides of the kink;
  - ensemble averages (Eq. 31): within 3 combined standard errors.
"""
import math

import numpy as np
import pytest

import gpu_common as gc

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


def test_philox_bitexact(E, orc):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xffffffff
    eng = E.Engine(0, E.make_params(gamma=1.0), seed=0)
    try:
        for seed in (0, 5, 0xDEADBEEFCAFEF00D, 2 ** 64 - 1):
            got = eng.philox_words(ctr, seed)
            key = [seed & 0xffffffff, seed >> 32]
            for i in range(0, len(ctr), 7):
                assert list(got[i]) == orc.philox4x32_10(list(ctr[i]), key), (seed, i)
    finally:
        eng.close()


def test_philox_bitexact_million(E, orc):
    """10^6 (key, counter) pairs: random counters, the all-zero and all-one
    counters, and the stream contract's tag and index-carry edges."""
    rng = np.random.default_rng(21)
    ctr = rng.integers(0, 2 ** 32, size=(500000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xffffffff
    ctr[2:6, 1] = np.array([0, 1, 2, 3], dtype=np.uint32) << 30        # the four tags, point 0
    ctr[6:10, 0] = 0xffffffff                                         # index low word at its top
    eng = E.Engine(0, E.make_params(gamma=1.0), seed=0)
    try:
        for seed in (0x0123456789ABCDEF, 2 ** 64 - 1):
            got = eng.philox_words(ctr, seed)
            want = orc.philox_many(ctr, [seed & 0xffffffff, seed >> 32])
            assert np.array_equal(got, want), seed
    finally:
        eng.close()


def _cases(W):
    pois = W.poisson_point()
    dich = W.dichot_point()
    both = dict(pois, Fa=0.5, Fb=0.5, mua=2.0, mub=2.0, noise_flags=7)
    return {
        "inertial-poisson": (0, pois, W.period_steps(4.9, 100)),
        "inertial-dichot": (0, dich, W.period_steps(4.9, 200)),
        "inertial-all-noises": (0, both, W.period_steps(4.9, 100)),
        "inertial-gauss-normal": (0, dict(pois, noise_flags=1 | 2 | 8), W.period_steps(4.9, 100)),
        "inertial-compensated": (0, dict(pois, noise_flags=1 | 2 | 16), W.period_steps(4.9, 100)),
        "overdamped-washboard": (1, dict(pois, V0=0.2, a=0.5, Q=0.05, Fa=0.3, Fb=0.6, mua=2.0,
                                         mub=1.0, noise_flags=7), 0.002),
        "pwl-model-I-II": (2, dict(pois, V0=1.0, a=0.0, F=0.0, Q=0.01, zeta=0.667, Fa=3.0, Fb=1.1,
                                   mua=1.0, mub=0.3667, x0_lo=-1.0, x0_hi=1.0, noise_flags=7,
                                   **{"lambda": 2.25}), 0.001),
        # the dichotomous force as a drift term (SDE_DICHOT_IN_DRIFT)
        "inertial-dichot-drift": (0, dict(dich, noise_flags=1 | 4 | 32), W.period_steps(4.9, 200)),
        "inertial-all-drift": (0, dict(both, noise_flags=7 | 32), W.period_steps(4.9, 100)),
        "pwl-model-II-drift": (2, dict(pois, V0=1.0, a=0.0, F=0.0, Q=0.01, Fa=3.0, Fb=1.1, mua=1.0,
                                       mub=0.3667, x0_lo=-1.0, x0_hi=1.0, noise_flags=1 | 4 | 32),
                               0.001),
    }


@pytest.mark.parametrize("case", ["inertial-poisson", "inertial-dichot", "inertial-all-noises",
                                  "inertial-gauss-normal", "inertial-compensated",
                                  "overdamped-washboard", "pwl-model-I-II", "inertial-dichot-drift",
                                  "inertial-all-drift", "pwl-model-II-drift"])
@pytest.mark.parametrize("n_tr,n_avg", [(0, 32), (37, 27), (5, 59), (0, 64)])
def test_per_path_short_horizon(E, W, orc, case, n_tr, n_avg):
    model, prm, dt = _cases(W)[case]
    paths = 1000                      # 31 full tiles and a ragged one of 8 paths
    g_st, g = gc.engine_run(E, torch, model, prm, 11, paths, dt, n_tr, n_avg)
    r = orc.run_paths(model, gc.oracle_params(orc, prm), 11, 0, paths, dt, n_tr, n_avg)
    ok, n_excl = gc.events_equal(g, r)
    assert ok and n_excl == 0
    keep = r["kink_min"] > 1e-5
    assert keep.sum() >= 0.9 * paths
    dX = np.abs(g["X_f"] - r["X_f"])[keep]
    assert dX.max() <= 2e-5, (case, np.quantile(dX, [0.5, 0.99, 1.0]))
    if model == 0:
        dv = np.abs(g["v_f"].astype(np.float64) - r["v_f"])[keep]
        assert dv.max() <= 2e-4, (case, np.quantile(dv, [0.5, 0.99, 1.0]))
    dvb = np.abs(g["vbar"] - r["vbar"])[keep] * (n_avg * dt)
    assert dvb.max() <= 4e-5
    assert g_st["n"] == paths
    # the device FP64 sums equal the sums of the device per-path values
    assert abs(g_st["sums"][1] - math.fsum(g["vbar"])) <= 1e-12 * (1 + np.abs(g["vbar"]).sum())


@pytest.mark.parametrize("case,n", [("inertial-poisson", 100), ("inertial-dichot", 200),
                                    ("inertial-all-noises", 100), ("overdamped-washboard", 800)])
def test_per_path_one_drive_period(E, W, orc, case, n):
    """Per path over one drive period (spp steps; 800 steps of the overdamped
    washboard, which is not chaotic): |dX| <= 1e-4 and |dv| <= 1e-3.  The
    driven inertial washboard is chaotic: FP32 rounding grows by about e^{8}
    over a period (measured maxima 5.7e-5 in X and 3.0e-4 in v over 1000
    paths) and reaches O(1) by eight periods, where only the ensemble
    averages can be compared."""
    model, prm, dt = _cases(W)[case]
    paths = 1000
    _, g = gc.engine_run(E, torch, model, prm, 11, paths, dt, 0, n)
    r = orc.run_paths(model, gc.oracle_params(orc, prm), 11, 0, paths, dt, 0, n)
    ok, n_excl = gc.events_equal(g, r)
    assert ok and n_excl == 0
    dX = np.abs(g["X_f"] - r["X_f"])
    assert dX.max() <= 1e-4, (case, np.quantile(dX, [0.5, 0.99, 1.0]))
    if model == 0:
        dv = np.abs(g["v_f"].astype(np.float64) - r["v_f"])
        assert dv.max() <= 1e-3, (case, np.quantile(dv, [0.5, 0.99, 1.0]))


@pytest.mark.parametrize("case", ["inertial-poisson", "inertial-dichot", "pwl-model-I-II"])
def test_event_indices_long_horizon(E, W, orc, case):
    """Event streams do not depend on the dynamics: bit-exact at any horizon."""
    model, prm, dt = _cases(W)[case]
    paths, n = 512, 44000
    _, g = gc.engine_run(E, torch, model, prm, 3, paths, dt, 1000, n - 1000)
    r = orc.run_paths(model, gc.oracle_params(orc, prm), 3, 0, paths, dt, 1000, n - 1000)
    ok, n_excl = gc.events_equal(g, r)
    assert ok and n_excl <= 1
    assert g["jP"].mean() + g["jD"].mean() > 50        # many events per path


def test_ensemble_poisson_1024(E, W, orc):
    """The 1024-path Poisson workload in full (100 + 400 periods)."""
    s = W.run_spec("poisson_1024")
    g_st, g = gc.engine_run(E, torch, s["model"], s["params"], s["seed"], s["paths"], s["dt"],
                            s["n_transient"], s["n_avg"])
    r = orc.run_paths(s["model"], gc.oracle_params(orc, s["params"]), s["seed"], 0, s["paths"],
                      s["dt"], s["n_transient"], s["n_avg"])
    o = orc.stats(r, s["n_avg"])
    assert abs(g_st["mean_v"] - o["mean_v"]) <= gc.combined_tol(g_st, o)
    ok, _ = gc.events_equal(g, r)
    assert ok
    # time-and-ensemble velocity moments
    se_t = np.std(r["sum_v"] / s["n_avg"], ddof=1) / math.sqrt(s["paths"])
    assert abs(g_st["tmean_v"] - o["tmean_v"]) <= 3 * math.sqrt(2) * se_t
    assert abs(g_st["tvar_v"] / o["tvar_v"] - 1) < 0.02


def test_ensemble_dichot_full_size(E, W, orc):
    """The 2^20-path dichotomous workload at full size and horizon, in the launch
    shape the bench's autotuner picks (two paths per lane on packed FP32 pairs,
    flips drawn in windows, 64-thread blocks, persistent grid); every per-path
    result equals that of one path per lane bit for bit, and the oracle
    integrates 16384 of the same paths (about 30 s on 16 host cores).  Eq. 31's
    mean is compared twice: the GPU's over all 2^20 paths against the oracle's
    sample (3 combined standard errors, 2.9e-4, 0.9 % of <v>), and the GPU's
    over the same 16384 paths against the oracle's (the same noise
    realisations, which FP32 and FP64 arithmetic follow apart over 2200 drive
    periods, so again 3 combined standard errors, 4.0e-4)."""
    s = W.run_spec("dichot_2p20")
    g_st, g = gc.engine_run(E, torch, s["model"], s["params"], s["seed"], s["paths"], s["dt"],
                            s["n_transient"], s["n_avg"], tuning=(64, 0), ppt=2)
    one_st, one = gc.engine_run(E, torch, s["model"], s["params"], s["seed"], s["paths"], s["dt"],
                                s["n_transient"], s["n_avg"])
    assert g_st["sums"] == one_st["sums"]
    for k in g:
        assert np.array_equal(g[k], one[k]), k
    assert g_st["n"] == s["paths"]
    sample = 16384
    first = s["paths"] - sample           # the last tiles of the launch
    r = orc.run_paths(s["model"], gc.oracle_params(orc, s["params"]), s["seed"], first, sample,
                      s["dt"], s["n_transient"], s["n_avg"])
    o = orc.stats(r, s["n_avg"])
    assert abs(g_st["mean_v"] - o["mean_v"]) <= gc.combined_tol(g_st, o)
    vb = g["vbar"][first:]
    same = {"mean_v": float(vb.mean()), "stderr_v": float(vb.std(ddof=1) / math.sqrt(sample))}
    assert abs(same["mean_v"] - o["mean_v"]) <= gc.combined_tol(same, o)
    assert gc.combined_tol(same, o) < 0.015 * abs(o["mean_v"])      # the bar has power
    keep = r["evt_margin"] > 1e-9
    np.testing.assert_array_equal(g["jD"][first:][keep].astype(np.uint64), r["jD"][keep])
    assert np.isfinite(g["X_f"]).all()


def test_models_against_oracle_ensemble(E, W, orc):
    """Overdamped washboard (Stratonovich regime) and Model II (Eq. 21b)."""
    import closed_forms as cf
    prm = dict(V0=1.0, F=5.0, Q=1.0, x0_hi=1.0, noise_flags=1)
    g_st, _ = gc.engine_run(E, torch, 1, prm, 0, 8192, 0.002, 2000, 20000, per_path=False)
    want = cf.stratonovich_velocity(1.0, 5.0, 1.0)
    assert abs(g_st["mean_v"] - want) < 4 * g_st["stderr_v"] + 0.015
    Fa, Fb, tau = 3.0, 1.1, 1.0
    mua, mub = Fa / (tau * (Fa + Fb)), Fb / (tau * (Fa + Fb))
    dt = min(1 / mua, 1 / mub) / 200
    n = int(400 * min(1 / mua, 1 / mub) / dt)
    prm = dict(Fa=Fa, Fb=Fb, mua=mua, mub=mub, x0_lo=-1.0, x0_hi=1.0, noise_flags=4)
    g_st, _ = gc.engine_run(E, torch, 2, prm, 0, 8192, dt, n // 10, n - n // 10, per_path=False)
    assert abs(g_st["mean_v"] - cf.eq21b_velocity(Fa, Fb, tau)) < 4 * g_st["stderr_v"] + 0.005


@pytest.mark.parametrize("case", ["inertial-dichot-drift", "pwl-model-II-drift"])
def test_dichotomous_drift_ensemble(E, W, orc, case):
    """Ensemble parity of the drift variant over a long horizon (22,000 steps),
    with the dichotomous flips bit-exact."""
    model, prm, dt = _cases(W)[case]
    paths, n_tr, n_avg = 2048, 2000, 20000
    g_st, g = gc.engine_run(E, torch, model, prm, 6, paths, dt, n_tr, n_avg)
    r = orc.run_paths(model, gc.oracle_params(orc, prm), 6, 0, paths, dt, n_tr, n_avg)
    o = orc.stats(r, n_avg)
    assert abs(g_st["mean_v"] - o["mean_v"]) <= gc.combined_tol(g_st, o)
    ok, n_excl = gc.events_equal(g, r)
    assert ok and n_excl <= 2


def test_launch_shape_does_not_change_results(E, W):
    s = W.run_spec("poisson_1024")
    ref = None
    for tuning in [(128, 0), (64, 0), (32, 3), (96, 1), (128, 1000)]:
        st, g = gc.engine_run(E, torch, s["model"], s["params"], 1, 2000, s["dt"], 333, 1000,
                              tuning=tuning)
        cur = (st["sums"], g["X_f"].tobytes(), g["jP"].tobytes())
        if ref is None:
            ref = cur
        assert cur == ref, tuning


def test_reduce_f64(E):
    eng = E.Engine(0, E.make_params(gamma=1.0), seed=0)
    try:
        rng = np.random.default_rng(4)
        for n in (1, 31, 32, 33, 4097, 1000003):
            x = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
            t = torch.from_numpy(x).cuda()
            cnt, s, s2 = eng.reduce_f64(t)
            assert cnt == n
            assert abs(s - math.fsum(x)) <= 1e-12 * np.abs(x).sum()
            assert abs(s2 - math.fsum(x * x)) <= 1e-12 * (x * x).sum()
    finally:
        eng.close()


def test_edge_sizes(E, W, orc):
    """One path (one lane of one tile), a single averaged step, no transient."""
    model, prm, dt = _cases(W)["inertial-all-noises"]
    for paths, n_tr, n_avg in ((1, 0, 1), (1, 3, 1), (33, 0, 2), (64, 31, 33)):
        st, g = gc.engine_run(E, torch, model, prm, 2, paths, dt, n_tr, n_avg)
        r = orc.run_paths(model, gc.oracle_params(orc, prm), 2, 0, paths, dt, n_tr, n_avg)
        assert st["n"] == paths
        assert np.abs(g["X_f"] - r["X_f"]).max() <= 2e-5
        ok, _ = gc.events_equal(g, r)
        assert ok


def test_invalid_arguments(E):
    eng = E.Engine(0, E.make_params(gamma=1.0), seed=0)
    try:
        with pytest.raises(E.SdeError) as ei:
            eng.stats()
        assert ei.value.code == E.SDE_ESTATE
        for args in ((0, 0.01, 0, 10), (10, 0.0, 0, 10), (10, float("nan"), 0, 10),
                     (10, 0.01, 0, 0), (10, 0.01, 2 ** 32, 10), (2 ** 33, 0.01, 0, 10)):
            with pytest.raises(E.SdeError) as ei:
                eng.run(*args)
            assert ei.value.code == E.SDE_EINVAL, args
        with pytest.raises(E.SdeError):
            eng.set_params(E.make_params(gamma=float("nan")))
        with pytest.raises(E.SdeError):
            eng.set_tuning(48, 0)
    finally:
        eng.close()
    with pytest.raises(E.SdeError):
        E.Engine(0, E.make_params(gamma=0.0), seed=0)
    with pytest.raises(E.SdeError):
        E.Engine(0, E.make_params(gamma=1.0, noise_flags=2), seed=0)   # Poisson needs lambda, zeta
