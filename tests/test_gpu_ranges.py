"""GPU tests of sde_run_range: disjoint path ranges of one ensemble (the
multi-GPU partition, emulated on one GPU one range after another) give the
per-path results of one run over their union bit for bit, and their five FP64
sums add up to its sums."""
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


def _run(E, prm, seed, first, paths, dt, n_tr, n_avg, ppt=1, steps_per_launch=0):
    eng = E.Engine(0, E.make_params(**prm), seed=seed)
    try:
        eng.set_paths_per_thread(ppt)
        eng.set_steps_per_launch(steps_per_launch)
        out = {"X_f": torch.zeros(paths, dtype=torch.float64, device="cuda"),
               "vbar": torch.zeros(paths, dtype=torch.float64, device="cuda"),
               "jD": torch.zeros(paths, dtype=torch.int32, device="cuda"),
               "jP": torch.zeros(paths, dtype=torch.int32, device="cuda")}
        eng.run(paths, dt, n_tr, n_avg, path_out=out, first_path=first)
        st = eng.stats()
    finally:
        eng.close()
    return st, {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("workload,ppt,spl", [("dichot_2p20", 2, 0), ("poisson_1024", 1, 0),
                                             ("dichot_2p20", 1, 1024)])
def test_ranges_equal_one_run(E, workload, ppt, spl):
    from paper_1409_4923_gb300 import workloads as W
    s = W.run_spec(workload)
    N, cut, n_tr, n_avg = 3000, 1344, 700, 3300          # ragged: the cut is a multiple of 32 + 0
    whole_st, whole = _run(E, s["params"], 5, 0, N, s["dt"], n_tr, n_avg, ppt, spl)
    a_st, a = _run(E, s["params"], 5, 0, cut, s["dt"], n_tr, n_avg, ppt, spl)
    b_st, b = _run(E, s["params"], 5, cut, N - cut, s["dt"], n_tr, n_avg, ppt, spl)
    for k in whole:
        np.testing.assert_array_equal(np.concatenate([a[k], b[k]]), whole[k], err_msg=k)
    comb = [x + y for x, y in zip(a_st["sums"], b_st["sums"])]
    assert comb[0] == whole_st["sums"][0] == N
    for x, y in zip(comb[1:], whole_st["sums"][1:]):
        assert abs(x - y) <= 1e-12 * abs(y)


def test_range_against_oracle(E, orc):
    """A range far from path 0 draws the oracle's random numbers for those paths."""
    from paper_1409_4923_gb300 import workloads as W
    s = W.run_spec("poisson_1024")
    first, n, n_tr, n_avg = 1000003, 96, 0, 64          # the per-path bar of 64 steps
    st, g = _run(E, s["params"], 2, first, n, s["dt"], n_tr, n_avg)
    r = orc.run_paths(s["model"], gc.oracle_params(orc, s["params"]), 2, first, n, s["dt"], n_tr, n_avg)
    ok, n_excl = gc.events_equal(g, r)
    assert ok and n_excl <= 1
    assert np.max(np.abs(g["X_f"] - r["X_f"])) < 2e-5


def test_range_limits(E):
    from paper_1409_4923_gb300 import workloads as W
    s = W.run_spec("poisson_1024")
    eng = E.Engine(0, E.make_params(**s["params"]), seed=0)
    try:
        with pytest.raises(E.SdeError):
            eng.run(64, s["dt"], 0, 32, first_path=(1 << 32) - 32)
        eng.run(32, s["dt"], 0, 32, first_path=(1 << 32) - 32)        # the last whole tile
        assert eng.stats()["n"] == 32
    finally:
        eng.close()
