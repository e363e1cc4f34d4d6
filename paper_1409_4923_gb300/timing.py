"""Timings quoted in the engine's documentation, each one command on one GPU.

  python -m paper_1409_4923_gb300.timing scan_64x64      # the 64 x 64 Poisson scan
  python -m paper_1409_4923_gb300.timing dichot_reruns   # 256 dichotomous points x 8192 paths
  python -m paper_1409_4923_gb300.timing scan_64x64 --mode 1   # the persistent scan kernel
  python -m paper_1409_4923_gb300.timing point poisson_1024 --paths 1048576 --steps 16384

Scans: the scan autotuner's launch shape, in the mode sde_scan chooses (one
point-kernel launch per point on side streams when the points hold 2048 paths
or more on average, else one persistent launch whose graph the first
repetition captures and later ones replay), or the mode --mode asks for
(sde_set_scan_mode: 1 persistent, 2 one launch per point); wall time around the call, the
best of the repetitions.  Point runs: CUDA events around sde_run on the
engine's stream, the best of a few repetitions.  Orchestration only.
"""
import json
import time


def _scan_points(name, E, W):
    if name == "scan_64x64":
        pts = W.scan_64x64()
    else:                                   # the guided scan's re-run shape
        pts = []
        for i in range(256):
            prm = W.dichot_point(b=2.0 * i / 255, F=-0.3 + 0.6 * ((i * 37) % 256) / 255, point=i)
            pts.append(dict(params=prm, dt=W.period_steps(4.9, 200), paths=8192, n_transient=40000,
                            n_avg=400000))
    return [dict(p, params=E.make_params(**p["params"])) for p in pts]


def time_scan(name, reps=2, mode=0):
    import torch
    from . import autotune, engine as E, workloads as W
    arg = _scan_points(name, E, W)
    path_steps = float(sum(p["paths"] * (p["n_transient"] + p["n_avg"]) for p in arg))
    eng = E.Engine(0, arg[0]["params"], seed=0)
    try:
        knobs = autotune.tune_scan(0, arg)
        autotune.apply_tuning(eng, knobs)
        eng.set_scan_mode(mode)
        eng.scan([dict(p, n_transient=0, n_avg=256) for p in arg[:256]])          # warm-up
        times = []
        for _ in range(max(1, reps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = eng.scan(arg)
            times.append(time.perf_counter() - t0)
    finally:
        eng.close()
    t = min(times)
    return {"workload": name, "points": len(arg), "path_steps": path_steps, "seconds": t,
            "seconds_each": times, "path_steps_per_s": path_steps / t, "points_per_s": len(arg) / t,
            "launch_shape": knobs, "scan_mode": mode, "mean_v_first_last": [res[0]["mean_v"], res[-1]["mean_v"]]}


def time_point(workload, paths, steps, reps=5):
    import torch
    from . import autotune, engine as E, workloads as W
    s = W.run_spec(workload)
    prm = E.make_params(**s["params"])
    stream = torch.cuda.Stream()
    knobs = autotune.tune(s["model"], prm, s["dt"], paths, stream=stream)
    eng = E.Engine(s["model"], prm, seed=0, stream=stream)
    try:
        autotune.apply_tuning(eng, {k: knobs[k] for k in autotune.DEFAULT})
        eng.run(paths, s["dt"], 0, min(steps, 2048))
        eng.stats()
        times = []
        for _ in range(max(1, reps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eng.run(paths, s["dt"], 0, steps)
            e1.record(stream)
            eng.stats()
            times.append(e0.elapsed_time(e1) / 1e3)
    finally:
        eng.close()
    t = min(times)
    return {"workload": workload, "paths": paths, "steps": steps, "seconds": t,
            "path_steps_per_s": float(paths) * steps / t,
            "launch_knobs": {k: knobs[k] for k in autotune.DEFAULT}}


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="timings of the engine on one GPU")
    ap.add_argument("what", choices=["scan_64x64", "dichot_reruns", "point"])
    ap.add_argument("workload", nargs="?", default="poisson_1024")
    ap.add_argument("--paths", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=16384)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--mode", type=int, default=0, choices=[0, 1, 2], help="scans: 0 auto, 1 persistent, 2 per point")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.what == "point":
        print(json.dumps(time_point(a.workload, a.paths, a.steps, max(a.reps, 3))))
    else:
        print(json.dumps(time_scan(a.what, a.reps, a.mode)))


if __name__ == "__main__":
    main()
