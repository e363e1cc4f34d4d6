"""GPU tests: the launch knobs of the autotuner (threads per block, grid,
paths per lane, steps per launch) never change a result bit."""
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
    both = dict(pois, Fa=0.5, Fb=0.5, mua=2.0, mub=2.0, noise_flags=7)
    return [
        (0, both, W.period_steps(4.9, 100)),
        (0, dict(both, noise_flags=5), W.period_steps(4.9, 200)),
        (0, dict(both, noise_flags=3), W.period_steps(4.9, 100)),
        (0, dict(both, noise_flags=1 | 2 | 8), W.period_steps(4.9, 100)),
        (0, dict(both, noise_flags=6), W.period_steps(4.9, 100)),
        (0, dict(both, noise_flags=7 | 32), W.period_steps(4.9, 100)),
        (1, dict(pois, V0=0.2, a=0.5, Q=0.05, Fa=0.3, Fb=0.6, mua=2.0, mub=1.0, noise_flags=7), 0.002),
        (2, dict(pois, V0=1.0, a=0.0, F=0.0, Q=0.01, zeta=0.667, Fa=3.0, Fb=1.1, mua=1.0,
                 mub=0.3667, x0_lo=-1.0, x0_hi=1.0, noise_flags=7, **{"lambda": 2.25}), 0.001),
    ]


def _run(E, model, prm, paths, dt, n_tr, n_avg, ppt=1, tuning=None, spl=0):
    eng = E.Engine(model, E.make_params(**prm), seed=3)
    try:
        eng.set_paths_per_thread(ppt)
        if tuning:
            eng.set_tuning(*tuning)
        eng.set_steps_per_launch(spl)
        out = {"X_f": torch.zeros(paths, dtype=torch.float64, device="cuda"),
               "v_f": torch.zeros(paths, dtype=torch.float32, device="cuda"),
               "vbar": torch.zeros(paths, dtype=torch.float64, device="cuda"),
               "jP": torch.zeros(paths, dtype=torch.int32, device="cuda"),
               "jD": torch.zeros(paths, dtype=torch.int32, device="cuda")}
        eng.run(paths, dt, n_tr, n_avg, path_out=out)
        st = eng.stats()
    finally:
        eng.close()
    return st["sums"], {k: v.cpu().numpy() for k, v in out.items()}


def _same(a, b):
    assert a[0] == b[0]
    for k in a[1]:
        assert np.array_equal(a[1][k], b[1][k]), k


@pytest.mark.parametrize("idx", range(8))
@pytest.mark.parametrize("paths", [1, 33, 1000, 2048 + 32])   # 1 and 33 items: an odd item count
def test_two_paths_per_lane_is_bit_identical(E, W, idx, paths):
    model, prm, dt = _cases(W)[idx]
    ref = _run(E, model, prm, paths, dt, 37, 600)
    _same(_run(E, model, prm, paths, dt, 37, 600, ppt=2), ref)


def test_two_paths_per_lane_any_launch_shape(E, W):
    model, prm, dt = _cases(W)[1]
    ref = _run(E, model, prm, 3000, dt, 64, 700)
    for tuning in [(32, 1), (64, 0), (96, 5), (128, 1000)]:
        _same(_run(E, model, prm, 3000, dt, 64, 700, ppt=2, tuning=tuning), ref)


@pytest.mark.parametrize("spl", [32, 96, 1024])
def test_steps_per_launch_is_bit_identical(E, W, spl):
    for model, prm, dt in _cases(W)[::2] + _cases(W)[5:6]:
        ref = _run(E, model, prm, 1000, dt, 100, 900)
        _same(_run(E, model, prm, 1000, dt, 100, 900, spl=spl), ref)


def test_knob_validation(E, W):
    model, prm, dt = _cases(W)[0]
    eng = E.Engine(model, E.make_params(**prm), seed=3)
    try:
        for bad in (0, 3, -1):
            with pytest.raises(E.SdeError):
                eng.set_paths_per_thread(bad)
        for bad in (1, 33, 100):
            with pytest.raises(E.SdeError):
                eng.set_steps_per_launch(bad)
    finally:
        eng.close()


def test_scan_point_kernels_with_two_paths_per_lane(E, W):
    prm = dict(V0=1.0, F=2.0, Q=0.5, x0_hi=1.0, noise_flags=1)
    pts = [dict(params=E.make_params(**dict(prm, F=F, point=i)), dt=0.002, paths=300 + 70 * i,
                n_transient=100, n_avg=700) for i, F in enumerate((0.5, 2.0, 4.0))]
    res = []
    for ppt in (1, 2):
        eng = E.Engine(1, pts[0]["params"], seed=1)
        try:
            eng.set_paths_per_thread(ppt)
            res.append([r["sums"] for r in eng.scan(pts)])
        finally:
            eng.close()
    assert res[0] == res[1]
