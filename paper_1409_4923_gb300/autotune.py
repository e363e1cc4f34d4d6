"""Launch-shape autotuner of the path kernels.

The knobs are the threads per block (32 .. 128) and the grid (0 = one
persistent wave sized by the occupancy calculator, or a fixed multiple of the
SM count).  Results never depend on the shape (each 32-path warp item is
integrated identically wherever it runs), so the tuner only times: it runs a
short probe of the same kernel variant (same model and noise switches) for
each candidate, keeps the fastest, and caches it per (device, variant, size
class) in a JSON file.  Engine users apply it with `apply(engine, ...)`.
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
    out = []
    for b in BLOCKS:
        for g in GRID_MULTIPLES:
            out.append((b, g * sm_count))
    return out


def choose(timings):
    """The fastest (block, grid) of {(block, grid): seconds}; ties go to the
    earlier candidate (the default shape comes first)."""
    best, best_t = None, float("inf")
    for cand, t in timings.items():
        if t < best_t * (1.0 - 1e-9):
            best, best_t = cand, t
    return best


def tune(model, params, dt, paths, n_probe_steps=2048, seed=0, stream=None, cache=None, force=False,
         log=None):
    """Time every candidate shape on a probe of `paths` paths x n_probe_steps
    steps (CUDA events) and cache the best; returns (block, grid, timings)."""
    import torch
    cache = cache or cache_path()
    dev = torch.cuda.get_device_name(torch.cuda.current_device())
    k = key(dev, model, params.noise_flags, paths)
    data = _load(cache)
    if not force and k in data:
        b, g = data[k]["block"], data[k]["grid"]
        return b, g, None
    eng = E.Engine(model, params, seed=seed, stream=stream)
    try:
        _, sms = eng.occupancy(128)
        timings = {}
        eng.run(paths, dt, 0, n_probe_steps)         # warm-up (module load, workspace)
        eng.stats()
        for b, g in candidates(sms):
            eng.set_tuning(b, g)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            eng.run(paths, dt, 0, n_probe_steps)
            eng.stats()
            timings[(b, g)] = time.perf_counter() - t0
            if log:
                log("block %3d grid %5d: %.3f ms" % (b, g, timings[(b, g)] * 1e3))
        b, g = choose(timings)
    finally:
        eng.close()
    data = _load(cache)
    data[k] = {"block": b, "grid": g, "probe_paths": paths, "probe_steps": n_probe_steps,
               "seconds": {"%d,%d" % bg: t for bg, t in timings.items()}}
    _store(cache, data)
    return b, g, timings


def apply(engine, model, params, dt, paths, **kw):
    """Tune (or read the cache) and set the engine's launch shape."""
    b, g, _ = tune(model, params, dt, paths, **kw)
    engine.set_tuning(b, g)
    return b, g
