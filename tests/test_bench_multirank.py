"""bench.py on the CPU: the N > 1 timing path on two gloo ranks (the slowest
rank's time is what every rank reports, and the weak-scaling value counts all
ranks' work over that time), the N > 1 data path (disjoint path ranges of one
ensemble whose five FP64 sums, added over the ranks, equal one process's run
over all paths; the oracle stands in for the engine on the CPU), and the JSON
line of the reference arm (the FP64 oracle on the host cores)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 1.5 + rank                     # rank 1 is the slow one
        t = bench.reduce_max_over_ranks(local)
        out.put((rank, t, bench.weak_scaling_value(100.0, world, 4, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(abs(r[2] - 100.0 * 2 * 4 / 2.5) < 1e-12 for r in res)


PER_RANK, N_TR, N_AVG = 48, 200, 800


def _five_sums(r):
    return [float(len(r)), float(r["vbar"].sum()), float((r["vbar"] ** 2).sum()),
            float(r["sum_v"].sum()), float(r["sum_v2"].sum())]


def _shard_main(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    import bench
    import oracle
    from paper_1409_4923_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = W.run_spec("dichot_2p20")
        prm = dict(s["params"])
        prm["noise"] = prm.pop("noise_flags")
        first, n = bench.shard_range(PER_RANK, rank)
        r = oracle.run_paths(s["model"], oracle.make_params(**prm), s["seed"], first, n, s["dt"],
                             N_TR, N_AVG, nthreads=1)
        comb = bench.combine_sums(_five_sums(r))
        out.put((rank, first, comb, r["X_f"].tolist(), r["jD"].tolist()))
    finally:
        dist.destroy_process_group()


def test_path_shards_combine_into_one_ensemble():
    """Rank r integrates paths [r P, (r + 1) P) under the common seed; the ranks'
    per-path results are those of one run over all 2 P paths bit for bit, and
    the all-reduced five sums give its Eq. 31 statistics (to FP64 summation
    order)."""
    import math
    import numpy as np
    import torch.multiprocessing as mp
    import bench
    import oracle
    from paper_1409_4923_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = W.run_spec("dichot_2p20")
    prm = dict(s["params"])
    prm["noise"] = prm.pop("noise_flags")
    whole = oracle.run_paths(s["model"], oracle.make_params(**prm), s["seed"], 0, world * PER_RANK,
                             s["dt"], N_TR, N_AVG, nthreads=1)
    assert [r[1] for r in res] == [0, PER_RANK]                       # disjoint, contiguous
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res]), whole["X_f"])
    np.testing.assert_array_equal(np.concatenate([r[4] for r in res]), whole["jD"])
    want = _five_sums(whole)
    for _, _, comb, _, _ in res:                                       # every rank holds the total
        assert comb[0] == want[0]
        for a, b in zip(comb[1:], want[1:]):
            assert abs(a - b) <= 1e-12 * abs(b) + 1e-300
    st = bench.ensemble_stats(res[0][2], N_AVG)
    o = oracle.stats(whole, N_AVG)
    assert st["n"] == world * PER_RANK
    assert abs(st["mean_v"] - o["mean_v"]) <= 1e-12 * abs(o["mean_v"]) + 1e-15
    assert math.isclose(st["stderr_v"], o["stderr_v"], rel_tol=1e-9)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_max_over_ranks(3.25) == 3.25
    assert bench.weak_scaling_value(10, 1, 2, 4.0) == 5.0


def test_reference_arm_json_line():
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "path-steps/s" and line["value"] > 0
    assert line["config"]["workload"] == "dichot_2p20" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
