"""GPU tests of segmented runs, checkpoints and scan resumption.

A segmented run advances every path by a number of steps per launch and
keeps the path states in device memory between launches (the structure of
the paper's Algorithm 5); a checkpoint carries those states to host memory
and back.  With cut points at multiples of 32 steps or at n_transient the
arithmetic is that of one launch, so results must be bit-identical to
sde_run_paths; any cut point leaves the random events bit-identical, since
the streams are addressed by (seed, point, path, step or event index).
"""
import ctypes

import numpy as np
import pytest

import gpu_common as gc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HEADER = 224


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
    return {
        "inertial-all-noises": (0, both, W.period_steps(4.9, 100)),
        "inertial-dichot": (0, dict(both, noise_flags=5), W.period_steps(4.9, 200)),
        "inertial-gauss-normal": (0, dict(both, noise_flags=1 | 2 | 8), W.period_steps(4.9, 100)),
        "overdamped-washboard": (1, dict(pois, V0=0.2, a=0.5, Q=0.05, Fa=0.3, Fb=0.6, mua=2.0,
                                         mub=1.0, noise_flags=7), 0.002),
        "pwl-model-I-II": (2, dict(pois, V0=1.0, a=0.0, F=0.0, Q=0.01, zeta=0.667, Fa=3.0, Fb=1.1,
                                   mua=1.0, mub=0.3667, x0_lo=-1.0, x0_hi=1.0, noise_flags=7,
                                   **{"lambda": 2.25}), 0.001),
    }


def _out(paths):
    return {"X_f": torch.zeros(paths, dtype=torch.float64, device="cuda"),
            "v_f": torch.zeros(paths, dtype=torch.float32, device="cuda"),
            "vbar": torch.zeros(paths, dtype=torch.float64, device="cuda"),
            "jP": torch.zeros(paths, dtype=torch.int32, device="cuda"),
            "jD": torch.zeros(paths, dtype=torch.int32, device="cuda")}


def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _segmented(E, model, prm, seed, paths, dt, n_tr, n_avg, cuts, tuning=None):
    """Run in segments ending at the given cut points, then to the end."""
    eng = E.Engine(model, E.make_params(**prm), seed=seed)
    try:
        if tuning:
            eng.set_tuning(*tuning)
        eng.begin(paths, dt, n_tr, n_avg)
        done = 0
        for c in cuts:
            done = eng.advance(c - done)
            assert done == c
        out = _out(paths)
        assert eng.advance(0, path_out=out) == n_tr + n_avg
        st = eng.stats()
    finally:
        eng.close()
    return st, _np(out)


def _assert_identical(a, b):
    for k in ("X_f", "v_f", "vbar", "jP", "jD"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("case", ["inertial-all-noises", "inertial-dichot", "inertial-gauss-normal",
                                  "overdamped-washboard", "pwl-model-I-II"])
def test_segments_at_chunk_edges_equal_one_launch(E, W, case):
    model, prm, dt = _cases(W)[case]
    paths, n_tr, n_avg = 1000, 100, 900            # a ragged tile; n_transient not a multiple of 32
    ref_st, ref = gc.engine_run(E, torch, model, prm, 5, paths, dt, n_tr, n_avg)
    st, seg = _segmented(E, model, prm, 5, paths, dt, n_tr, n_avg, [64, 100, 352, 608, 640])
    _assert_identical(seg, ref)
    assert st["sums"] == ref_st["sums"]


def test_segments_do_not_depend_on_launch_shape(E, W):
    model, prm, dt = _cases(W)["inertial-all-noises"]
    _, a = _segmented(E, model, prm, 2, 777, dt, 64, 448, [96, 256])
    _, b = _segmented(E, model, prm, 2, 777, dt, 64, 448, [96, 256], tuning=(32, 7))
    _assert_identical(a, b)


def test_unaligned_cuts_keep_the_random_events(E, W):
    """Cut points inside a 32-step chunk fold x at other steps (FP32 rounding
    differs) but draw the same events; the ensemble mean agrees far inside
    its statistical error."""
    model, prm, dt = _cases(W)["inertial-all-noises"]
    paths, n_tr, n_avg = 4096, 300, 3000
    ref_st, ref = gc.engine_run(E, torch, model, prm, 8, paths, dt, n_tr, n_avg)
    st, seg = _segmented(E, model, prm, 8, paths, dt, n_tr, n_avg, [50, 77, 301, 1333, 2999])
    assert np.array_equal(seg["jP"], ref["jP"]) and np.array_equal(seg["jD"], ref["jD"])
    assert abs(st["mean_v"] - ref_st["mean_v"]) <= 0.1 * gc.combined_tol(st, ref_st)
    assert st["n"] == paths


@pytest.mark.parametrize("cut", [0, 352, 1000])
def test_checkpoint_restore_in_a_new_context(E, W, cut):
    """Checkpoint after `cut` steps (0: before any step; 1000: complete), restore
    into a context created with other parameters and another seed, finish:
    bit-identical to the uninterrupted run."""
    model, prm, dt = _cases(W)["inertial-all-noises"]
    paths, n_tr, n_avg = 1000, 100, 900
    ref_st, ref = gc.engine_run(E, torch, model, prm, 5, paths, dt, n_tr, n_avg)
    a = E.Engine(model, E.make_params(**prm), seed=5)
    try:
        a.begin(paths, dt, n_tr, n_avg)
        if cut:
            assert a.advance(cut) == cut
        blob = a.checkpoint()
    finally:
        a.close()
    assert len(blob) == HEADER + (84 * 1024 if cut else 0)
    b = E.Engine(model, E.make_params(**dict(prm, F=-0.2, Q=0.01)), seed=123)
    try:
        b.restore(blob)
        out = _out(paths)
        assert b.advance(0, path_out=out) == n_tr + n_avg
        st = b.stats()
        # the context's own parameters and seed are untouched by the restore
        b.run(64, dt, 0, 64)
        assert b.stats()["n"] == 64
    finally:
        b.close()
    _assert_identical(_np(out), ref)
    assert st["sums"] == ref_st["sums"]


def _fnv1a64(data):
    h = 0xcbf29ce484222325
    for byte in data:
        h ^= byte
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def test_restore_rejects_bad_checkpoints(E, W):
    model, prm, dt = _cases(W)["inertial-all-noises"]
    a = E.Engine(model, E.make_params(**prm), seed=5)
    try:
        with pytest.raises(E.SdeError) as ei:
            a.advance(10)
        assert ei.value.code == E.SDE_ESTATE
        with pytest.raises(E.SdeError) as ei:
            a.checkpoint()
        assert ei.value.code == E.SDE_ESTATE
        a.begin(100, dt, 40, 200)
        a.advance(96)
        good = a.checkpoint()
    finally:
        a.close()
    stride = 128
    assert len(good) == HEADER + 84 * stride
    bad = []
    flipped = bytearray(good)
    flipped[HEADER + 1000] ^= 1                               # state byte: checksum
    bad.append(bytes(flipped))
    bad.append(good[:-1])                                     # truncated
    bad.append(good[:100])                                    # shorter than the header
    bad.append(b"X" + good[1:])                               # magic
    forged = bytearray(good)                                  # eP of path 0 < steps done,
    forged[HEADER + 44 * stride:HEADER + 44 * stride + 4] = (5).to_bytes(4, "little")
    forged[216:224] = _fnv1a64(forged[HEADER:]).to_bytes(8, "little")   # with a valid checksum
    bad.append(bytes(forged))
    for blob in bad:
        b = E.Engine(model, E.make_params(**prm), seed=5)
        try:
            with pytest.raises(E.SdeError) as ei:
                b.restore(blob)
            assert ei.value.code == E.SDE_EINVAL
            with pytest.raises(E.SdeError):                   # nothing was restored
                b.advance(0)
        finally:
            b.close()
    other = E.Engine(1, E.make_params(**dict(prm, V0=0.2)), seed=5)   # another model
    try:
        with pytest.raises(E.SdeError) as ei:
            other.restore(good)
        assert ei.value.code == E.SDE_EINVAL
    finally:
        other.close()
    # the forged file differs from the good one only in the event counter
    ok = E.Engine(model, E.make_params(**prm), seed=5)
    try:
        ok.restore(good)
        assert ok.advance(0) == 240
    finally:
        ok.close()


def _scan_points(E, W, n, paths, n_avg):
    return [dict(params=E.make_params(**dict(W.poisson_point(F=-0.3 + 0.6 * i / max(n - 1, 1)),
                                             point=i)),
                 dt=W.period_steps(4.9, 100), paths=paths, n_transient=100, n_avg=n_avg)
            for i in range(n)]


def test_scan_resume_equals_uninterrupted(E, W):
    pts = _scan_points(E, W, 16, 2048, 2000)          # 1024 items
    eng = E.Engine(0, pts[0]["params"], seed=4)
    try:
        eng.set_scan_mode(1)                          # the persistent scan kernel
        ref = eng.scan(pts)
        eng.set_tuning(32, 152)                       # 152 warps: about 152 items per launch
        calls = 1
        try:
            res = eng.scan(pts, deadline_ms=0.001)
            pytest.fail("the scan should have run out of time")
        except E.SdeTimeout:
            pass
        while True:
            calls += 1
            assert calls < 100
            try:
                res = eng.scan_resume(deadline_ms=0.001)
                break
            except E.SdeTimeout:
                continue
        assert calls >= 3
        with pytest.raises(E.SdeError) as ei:          # nothing left to resume
            eng.scan_resume()
        assert ei.value.code == E.SDE_ESTATE
    finally:
        eng.close()
    for r, q in zip(res, ref):
        assert r["sums"] == q["sums"] and r["status"] == 0


def test_scan_resume_point_kernels_and_invalidation(E, W):
    prm = dict(V0=1.0, F=2.0, Q=0.5, x0_hi=1.0, noise_flags=1)
    pts = [dict(params=E.make_params(**dict(prm, F=F, point=i)), dt=0.002, paths=600,
                n_transient=100, n_avg=700) for i, F in enumerate((0.5, 2.0, 4.0))]
    eng = E.Engine(1, pts[0]["params"], seed=1)
    try:
        ref = eng.scan(pts)
        eng.set_tuning(32, 2)                         # 2 warps per point launch
        with pytest.raises(E.SdeTimeout):
            eng.scan(pts, deadline_ms=0.001)
        res = eng.scan_resume()                       # no deadline: finishes
        for r, q in zip(res, ref):
            assert r["sums"] == q["sums"]
        with pytest.raises(E.SdeTimeout):
            eng.scan(pts, deadline_ms=0.001)
        eng.run(64, 0.002, 0, 64)                     # reuses the workspace
        eng.stats()
        with pytest.raises(E.SdeError) as ei:
            eng.scan_resume()
        assert ei.value.code == E.SDE_ESTATE
    finally:
        eng.close()
