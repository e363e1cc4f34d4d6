"""Launch autotuner of the path kernels.

Knobs: threads per block (32 .. 128), the grid (0 = one persistent wave sized
by the occupancy calculator, or a fixed multiple of the SM count), paths per
lane (1 or 2, interleaved) and steps per launch (0 = the whole run in one
launch, or Algorithm 5's `samples` steps per launch with the path states kept
in device memory between launches).  `tune` serves single-point runs,
`tune_scan` the batched scan (block and grid).  Results never depend on any of them (each
path takes the same operations however it is scheduled; the tests check this
bit for bit), so the tuner only times: it runs a short probe of the same
kernel variant (same model and noise switches) for each candidate, keeps the
fastest, and caches it per (device, variant, size class) in a JSON file.
Engine users apply it with `apply(engine, ...)`.
"""
import json
import math
import os
import time

from . import engine as E

CACHE_ENV = "SDE_AUTOTUNE_CACHE"
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sde_gb300", "autotune.json")

BLOCKS = (32, 64, 96, 128)
GRID_MULTIPLES = (0, 1, 2, 4)         # 0: persistent full-occupancy wave; k: k x SMs blocks
PATHS_PER_THREAD = (1, 2)
STEPS_PER_LAUNCH = (0, 1024)          # 0: whole run per launch
DEFAULT = {"block": 128, "grid": 0, "ppt": 1, "steps_per_launch": 0}


def cache_path():
    return os.environ.get(CACHE_ENV, DEFAULT_CACHE)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def size_class(paths):
    """Bucket of the path count (powers of four) so that one tuning serves similar runs."""
    return int(math.log(max(paths, 1), 4))


def key(device_name, model, flags, paths):
    return "%s|model=%d|flags=%d|paths~4^%d" % (device_name, model, flags, size_class(paths))


def candidates(sm_count):
    """(block, grid, paths per thread) shapes; the default comes first."""
    out = []
    for ppt in PATHS_PER_THREAD:
        for b in sorted(BLOCKS, reverse=True):
            for g in GRID_MULTIPLES:
                out.append((b, g * sm_count, ppt))
    return out


def choose(timings):
    """The fastest candidate of {candidate: seconds}; ties go to the earlier
    candidate (the default comes first)."""
    best, best_t = None, float("inf")
    for cand, t in timings.items():
        if t < best_t * (1.0 - 1e-9):
            best, best_t = cand, t
    return best


def _time_run(eng, paths, dt, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng.run(paths, dt, 0, steps)
    eng.stats()
    return time.perf_counter() - t0


def tune(model, params, dt, paths, n_probe_steps=2048, seed=0, stream=None, cache=None, force=False,
         log=None):
    """Time every candidate on a probe of `paths` paths x n_probe_steps steps
    (shape stage), then the steps-per-launch candidates on 2 x n_probe_steps
    steps with the best shape; caches and returns a dict with keys block,
    grid, ppt, steps_per_launch (and seconds, the probe timings, when it ran)."""
    import torch
    cache = cache or cache_path()
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    k = key(dev, model, params.noise_flags, paths)
    data = _load(cache)
    if not force and k in data and all(f in data[k] for f in DEFAULT):
        return {f: data[k][f] for f in DEFAULT}
    eng = E.Engine(model, params, seed=seed, stream=stream)
    try:
        _, sms = eng.occupancy(128)
        eng.run(paths, dt, 0, n_probe_steps)         # warm-up (module load, workspace)
        eng.stats()
        shapes = {}
        for b, g, ppt in candidates(sms):
            eng.set_paths_per_thread(ppt)
            eng.set_tuning(b, g)
            shapes[(b, g, ppt)] = _time_run(eng, paths, dt, n_probe_steps)
            if log:
                log("block %3d grid %5d ppt %d: %.3f ms" % (b, g, ppt, shapes[(b, g, ppt)] * 1e3))
        b, g, ppt = choose(shapes)
        eng.set_paths_per_thread(ppt)
        eng.set_tuning(b, g)
        spl = {}
        for s in STEPS_PER_LAUNCH:
            eng.set_steps_per_launch(s)
            _time_run(eng, paths, dt, 2 * n_probe_steps)          # allocates the saved states once
            spl[s] = _time_run(eng, paths, dt, 2 * n_probe_steps)
            if log:
                log("steps per launch %d: %.3f ms" % (s, spl[s] * 1e3))
        s = choose(spl)
    finally:
        eng.close()
    res = {"block": b, "grid": g, "ppt": ppt, "steps_per_launch": s}
    data = _load(cache)
    data[k] = dict(res, probe_paths=paths, probe_steps=n_probe_steps,
                   seconds={"%d,%d,%d" % c: t for c, t in shapes.items()},
                   seconds_steps_per_launch={str(c): t for c, t in spl.items()})
    _store(cache, data)
    return dict(res, seconds=shapes, seconds_steps_per_launch=spl)


def scan_key(device_name, model, flags, items):
    """Cache key of a scan shape: a shape tuned on a few hundred 32-path items
    (a fixed grid of one wave can win there) must not serve a scan of 10^5."""
    return "%s|scan|model=%d|flags=%d|items~4^%d" % (device_name, model, flags, size_class(items))


def tune_scan(model, points, seed=0, n_probe_points=256, probe_steps=4096, stream=None, cache=None,
              force=False, log=None):
    """Launch shape of the batched scan: time every (block, grid) candidate on a
    probe scan of the first n_probe_points points, each cut to probe_steps
    steps (one persistent launch per candidate), and cache the fastest per
    (device, model, noise flags, size class of the points' 32-path items).  Paths per lane and steps per launch do not
    apply to the scan kernel.  Returns dict(block, grid)."""
    import torch
    cache = cache or cache_path()
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    flags = points[0]["params"].noise_flags
    items = sum((int(p["paths"]) + 31) // 32 for p in points)
    k = scan_key(dev, model, flags, items)
    data = _load(cache)
    if not force and k in data:
        return {"block": data[k]["block"], "grid": data[k]["grid"]}
    probe = []
    for p in points[:n_probe_points]:
        n_tr = min(p["n_transient"], probe_steps // 4)
        probe.append(dict(p, n_transient=n_tr, n_avg=max(1, probe_steps - n_tr)))
    eng = E.Engine(model, points[0]["params"], seed=seed, stream=stream)
    try:
        _, sms = eng.occupancy(128)
        eng.scan(probe)                                  # warm-up (module load, workspace, graph)
        timings = {}
        for b, g, ppt in candidates(sms):
            if ppt != 1:
                continue
            eng.set_tuning(b, g)
            eng.scan(probe)                              # captures this shape's graph
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            eng.scan(probe)
            timings[(b, g)] = time.perf_counter() - t0
            if log:
                log("scan block %3d grid %5d: %.3f ms" % (b, g, timings[(b, g)] * 1e3))
        b, g = choose(timings)
    finally:
        eng.close()
    data = _load(cache)
    data[k] = {"block": b, "grid": g, "probe_points": len(probe), "probe_steps": probe_steps,
               "seconds": {"%d,%d" % c: t for c, t in timings.items()}}
    _store(cache, data)
    return {"block": b, "grid": g}


def apply_tuning(engine, t):
    engine.set_tuning(t["block"], t["grid"])
    if "ppt" in t:
        engine.set_paths_per_thread(t["ppt"])
    if "steps_per_launch" in t:
        engine.set_steps_per_launch(t["steps_per_launch"])


def apply(engine, model, params, dt, paths, **kw):
    """Tune (or read the cache) and set the engine's launch knobs."""
    t = tune(model, params, dt, paths, **kw)
    apply_tuning(engine, t)
    return t
