"""The launch autotuner: selection, cache keys and the cache file (CPU), and one
real tuning on the GPU whose chosen knobs reproduce the default's results bit
for bit."""
import json

import pytest

from paper_1409_4923_gb300 import autotune as AT


def test_choose_picks_the_fastest_and_keeps_the_first_on_ties():
    t = {(128, 0, 1): 1.0, (64, 0, 1): 0.8, (32, 152, 2): 0.8, (96, 304, 1): 1.2}
    assert AT.choose(t) == (64, 0, 1)
    assert AT.choose({(128, 0, 1): 1.0, (64, 0, 1): 1.0}) == (128, 0, 1)
    assert AT.choose({0: 2.0, 1024: 2.5}) == 0


def test_candidates_and_keys():
    c = AT.candidates(152)
    assert c[0] == (128, 0, 1)                      # the default shape comes first
    assert (32, 608, 2) in c and len(set(c)) == len(c)
    assert len(c) == len(AT.BLOCKS) * len(AT.GRID_MULTIPLES) * len(AT.PATHS_PER_THREAD)
    assert AT.size_class(1 << 20) == 10 and AT.size_class(1) == 0
    assert AT.key("GB300", 0, 5, 1 << 20) != AT.key("GB300", 0, 6, 1 << 20)
    assert AT.key("GB300", 0, 5, 1 << 20) == AT.key("GB300", 0, 5, (1 << 20) + 5)
    assert all(s % 32 == 0 for s in AT.STEPS_PER_LAUNCH) and AT.STEPS_PER_LAUNCH[0] == 0
    # a scan shape tuned on a few hundred items never serves a scan of 10^5 items
    assert AT.scan_key("GB300", 0, 3, 288) != AT.scan_key("GB300", 0, 3, 294912)
    assert AT.scan_key("GB300", 0, 3, 294912) == AT.scan_key("GB300", 0, 3, 300000)
    assert AT.scan_key("GB300", 0, 3, 288) != AT.scan_key("GB300", 0, 5, 288)


def test_tests_tune_into_a_private_cache():
    import os
    assert AT.cache_path() != AT.DEFAULT_CACHE
    assert os.environ.get(AT.CACHE_ENV) == AT.cache_path()


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    AT._store(p, {"k": {"block": 64, "grid": 0}})
    assert AT._load(p) == {"k": {"block": 64, "grid": 0}}
    assert AT._load(str(tmp_path / "missing.json")) == {}
    with open(p, "w") as f:
        f.write("{broken")
    assert AT._load(p) == {}


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import engine as E, workloads as W
    spec = W.run_spec("dichot_2p20")
    prm = E.make_params(**spec["params"])
    cache = str(tmp_path / "tune.json")
    t = AT.tune(spec["model"], prm, spec["dt"], 1 << 16, n_probe_steps=512, cache=cache)
    assert (t["block"], t["grid"], t["ppt"]) in t["seconds"]
    assert len(t["seconds"]) == len(AT.candidates(torch.cuda.get_device_properties(0).multi_processor_count))
    assert t["steps_per_launch"] in AT.STEPS_PER_LAUNCH
    assert json.load(open(cache))
    t2 = AT.tune(spec["model"], prm, spec["dt"], 1 << 16, cache=cache)
    assert t2 == {f: t[f] for f in AT.DEFAULT}
    sums = []
    for knobs in (AT.DEFAULT, t2):
        eng = E.Engine(spec["model"], prm, seed=0)
        AT.apply_tuning(eng, knobs)
        eng.run(5000, spec["dt"], 100, 700)
        sums.append(eng.stats()["sums"])
        eng.close()
    assert sums[0] == sums[1]


@pytest.mark.gpu
def test_tune_scan_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4923_gb300 import engine as E, workloads as W
    pts = [dict(p, params=E.make_params(**p["params"])) for p in W.scan_64x64()[:64]]
    cache = str(tmp_path / "tune.json")
    t = AT.tune_scan(0, pts, n_probe_points=32, probe_steps=1024, cache=cache)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert t["block"] in AT.BLOCKS and t["grid"] % sms == 0
    assert AT.tune_scan(0, pts, cache=cache) == t
    sums = []
    for knobs in (AT.DEFAULT, t):
        eng = E.Engine(0, pts[0]["params"], seed=2)
        AT.apply_tuning(eng, knobs)
        short = [dict(p, n_avg=500, n_transient=50) for p in pts[:16]]
        sums.append([r["sums"] for r in eng.scan(short)])
        eng.close()
    assert sums[0] == sums[1]

