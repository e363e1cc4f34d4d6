"""sde_run_noalloc, the entry point that allocates nothing.

Some callers cannot allocate device memory: code running under a memory pool
or arena that must own every allocation, real-time loops that may not call
cudaMalloc/cudaFree (both can synchronise the device), hosts that forbid
allocation after start-up.  For them the library keeps its scratch in one
fixed-size device array and the caller passes only the outputs.  This test
calls that entry point through the C ABI and checks its sums against those
of the regular entry point (sde_run + sde_stats) on two calls in a row, so the
second call also shows that the shared array is cleared between calls, and
it reads the device's free memory around warm calls, which must not move.  It
sits in a file of its own that pytest collects last.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib_and_engine():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import engine as E
    L = E.lib()
    return L, E


def _reference_sums(E, model, prm, seed, paths, dt, n_tr, n_avg):
    eng = E.Engine(model, E.make_params(**prm), seed=seed)
    try:
        eng.run(paths, dt, n_tr, n_avg)
        return eng.stats()["sums"]
    finally:
        eng.close()


def test_noalloc_matches_regular_entry_point_twice():
    L, E = _lib_and_engine()
    from paper_1409_4923_gb300 import workloads as W
    cases = [(W.poisson_point(), W.period_steps(4.9, 100), 1000, 37, 2000, 3),     # ragged tile
             (W.dichot_point(), W.period_steps(4.9, 200), 4096, 0, 3200, 5)]
    out5 = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    for prm, dt, paths, n_tr, n_avg, seed in cases:        # two calls in a row
        want = _reference_sums(E, 0, prm, seed, paths, dt, n_tr, n_avg)
        p = E.make_params(**prm)
        rc = L.sde_run_noalloc(0, ctypes.byref(p), seed, paths, dt, n_tr, n_avg, None,
                               ctypes.c_void_p(out5.data_ptr()), ctypes.c_void_p(status.data_ptr()))
        assert rc == E.SDE_OK, L.sde_last_error(None)
        torch.cuda.synchronize()
        got = out5.cpu().tolist()
        assert got[0] == paths
        for g, w in zip(got, want):
            assert abs(g - w) <= 1e-12 * (1.0 + abs(w)), (got, want)
        assert int(status.item()) == E.SDE_OK


def test_noalloc_rejects_more_paths_than_its_scratch_holds():
    L, E = _lib_and_engine()
    from paper_1409_4923_gb300 import workloads as W
    out5 = torch.zeros(5, dtype=torch.float64, device="cuda")
    p = E.make_params(**W.poisson_point())
    rc = L.sde_run_noalloc(0, ctypes.byref(p), 0, E.NOALLOC_MAX_PATHS + 1, 0.01, 0, 10, None,
                           ctypes.c_void_p(out5.data_ptr()), None)
    assert rc == E.SDE_EINVAL
    assert b"SDE_NOALLOC_MAX_PATHS" in L.sde_last_error(None)


def test_noalloc_warm_calls_leave_free_device_memory_unchanged():
    """What the entry point is for: after the first call on the device (which
    loads the library's device code and creates the scratch array), further
    calls take no device memory.  cudaMemGetInfo's free bytes, read around
    three calls of the same kind, do not move."""
    L, E = _lib_and_engine()
    from paper_1409_4923_gb300 import workloads as W
    out5 = torch.zeros(5, dtype=torch.float64, device="cuda")
    p = E.make_params(**W.dichot_point())
    dt = W.period_steps(4.9, 200)

    def call():
        rc = L.sde_run_noalloc(0, ctypes.byref(p), 1, 8192, dt, 64, 512, None,
                               ctypes.c_void_p(out5.data_ptr()), None)
        assert rc == E.SDE_OK, L.sde_last_error(None)
        torch.cuda.synchronize()

    call()                                                  # first call: set-up
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert out5[0].item() == 8192
