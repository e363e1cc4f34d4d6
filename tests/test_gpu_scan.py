"""GPU tests of the batched scan (one persistent launch over many points) and
of the device-side deadline."""
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


def _points(E, W, flags=None):
    rng = np.random.default_rng(7)
    pts = []
    for i in range(9):
        prm = W.poisson_point(F=float(rng.uniform(-0.3, 0.3)), Q=float(10 ** rng.uniform(-4, -1)),
                              point=i)
        if flags is not None:
            prm.update(Fa=0.5, Fb=0.5, mua=2.0, mub=2.0, noise_flags=flags)
        pts.append(dict(params=prm, dt=W.period_steps(4.9, 100), paths=int(rng.integers(1, 700)),
                        n_transient=int(rng.integers(0, 300)), n_avg=int(rng.integers(1, 1500))))
    return pts


@pytest.mark.parametrize("flags", [None, 5, 7, 5 | 32])
def test_scan_equals_single_runs(E, W, flags):
    """Each point of a scan gives exactly (bitwise) the sums of its own run."""
    pts = _points(E, W, flags)
    eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=9)
    try:
        res = eng.scan([dict(p, params=E.make_params(**p["params"])) for p in pts])
        res2 = eng.scan([dict(p, params=E.make_params(**p["params"])) for p in pts])   # graph replay
    finally:
        eng.close()
    for p, r, r2 in zip(pts, res, res2):
        st, _ = gc.engine_run(E, torch, 0, p["params"], 9, p["paths"], p["dt"], p["n_transient"],
                              p["n_avg"], per_path=False)
        assert r["sums"] == st["sums"]
        assert r2["sums"] == st["sums"]
        assert r["n"] == p["paths"]


def test_scan_against_oracle(E, W, orc):
    pts = _points(E, W)
    eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=9)
    try:
        res = eng.scan([dict(p, params=E.make_params(**p["params"])) for p in pts])
    finally:
        eng.close()
    for p, r in zip(pts, res):
        o = orc.run_paths(0, gc.oracle_params(orc, p["params"]), 9, 0, p["paths"], p["dt"],
                          p["n_transient"], p["n_avg"])
        os_ = orc.stats(o, p["n_avg"])
        if p["paths"] > 1:
            assert abs(r["mean_v"] - os_["mean_v"]) <= gc.combined_tol(r, os_) + 1e-9


def test_scan_other_model_uses_point_kernels(E, W, orc):
    prm = dict(V0=1.0, F=2.0, Q=0.5, x0_hi=1.0, noise_flags=1)
    pts = [dict(params=dict(prm, F=F, point=i), dt=0.002, paths=300, n_transient=100, n_avg=700)
           for i, F in enumerate((0.5, 2.0, 4.0))]
    eng = E.Engine(1, E.make_params(**pts[0]["params"]), seed=1)
    try:
        res = eng.scan([dict(p, params=E.make_params(**p["params"])) for p in pts])
    finally:
        eng.close()
    for p, r in zip(pts, res):
        st, _ = gc.engine_run(E, torch, 1, p["params"], 1, p["paths"], p["dt"], p["n_transient"],
                              p["n_avg"], per_path=False)
        assert r["sums"] == st["sums"]


def test_deadline_times_out_and_context_survives(E, W):
    """A device budget far below the work: the kernel stops taking items, the
    host sees ETIMEDOUT, and the same context then runs normally."""
    pts = [dict(params=E.make_params(**W.poisson_point(point=i)), dt=W.period_steps(4.9, 100),
                paths=4096, n_transient=0, n_avg=200000) for i in range(64)]
    eng = E.Engine(0, pts[0]["params"], seed=0)
    try:
        with pytest.raises(E.SdeTimeout):
            eng.scan(pts, deadline_ms=0.001)
        eng.run(64, W.period_steps(4.9, 100), 0, 100)
        st = eng.stats()
        assert st["n"] == 64 and st["status"] == 0
        res = eng.scan(pts[:2], deadline_ms=0.0)
        assert all(r["status"] == 0 for r in res)
    finally:
        eng.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("flags", [None, 5])
def test_scan_device_outputs_equal_host_scan(E, W, flags, mode):
    """sde_scan_device leaves each point's five sums in a device array (no host
    round trip): the same values as sde_scan, bit for bit, also when the two
    calls alternate (each keeps its own captured graph), in both scan modes
    (the persistent kernel and one launch per point on side streams)."""
    pts = _points(E, W, flags)
    arg = [dict(p, params=E.make_params(**p["params"])) for p in pts]
    eng = E.Engine(0, arg[0]["params"], seed=4)
    try:
        eng.set_scan_mode(mode)
        out5 = torch.full((5 * len(arg),), float("nan"), dtype=torch.float64, device="cuda")
        eng.scan_device(arg, out5)
        host = eng.scan(arg)
        out5b = torch.zeros_like(out5)
        eng.scan_device(arg, out5b)
        torch.cuda.synchronize()
    finally:
        eng.close()
    d, db = out5.cpu().numpy().reshape(-1, 5), out5b.cpu().numpy().reshape(-1, 5)
    for i, h in enumerate(host):
        assert list(d[i]) == h["sums"]
        assert list(db[i]) == h["sums"]


@pytest.mark.parametrize("flags", [None, 5, 7])
def test_scan_modes_agree(E, W, flags):
    """The persistent scan kernel and one point-kernel launch per point (on side
    streams) give every point's sums bit for bit."""
    pts = _points(E, W, flags)
    arg = [dict(p, params=E.make_params(**p["params"])) for p in pts]
    res = {}
    for mode in (1, 2):
        eng = E.Engine(0, arg[0]["params"], seed=11)
        try:
            eng.set_scan_mode(mode)
            res[mode] = eng.scan(arg)
        finally:
            eng.close()
    for a, b in zip(res[1], res[2]):
        assert a["sums"] == b["sums"]
