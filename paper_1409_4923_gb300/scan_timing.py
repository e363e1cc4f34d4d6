"""Time the batched parameter scan of the Poisson model (64 x 64 grid of F and
log-spaced Q, path counts log-uniform in [256, 16384], averaged horizons
uniform in [500, 3000] drive periods; workloads.scan_64x64) as one persistent
launch on one GPU.

  python -m paper_1409_4923_gb300.scan_timing [--reps 2]

The launch shape comes from the scan autotuner; the first repetition
captures the scan graph, the later ones replay it.  Orchestration only.
"""
import json
import time


def main():
    import argparse
    import torch
    from . import autotune, engine as E, workloads as W
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    pts = W.scan_64x64()
    arg = [dict(p, params=E.make_params(**p["params"])) for p in pts]
    path_steps = float(sum(p["paths"] * (p["n_transient"] + p["n_avg"]) for p in pts))
    eng = E.Engine(0, arg[0]["params"], seed=0)
    try:
        knobs = autotune.tune_scan(0, arg)
        autotune.apply_tuning(eng, knobs)
        eng.scan([dict(p, n_transient=0, n_avg=256) for p in arg[:256]])          # warm-up
        times = []
        for _ in range(max(1, a.reps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = eng.scan(arg)
            times.append(time.perf_counter() - t0)
    finally:
        eng.close()
    t = min(times)
    print(json.dumps({"workload": "scan_64x64", "points": len(pts), "path_steps": path_steps,
                      "seconds": t, "seconds_each": times, "path_steps_per_s": path_steps / t,
                      "points_per_s": len(pts) / t, "launch_shape": knobs,
                      "mean_v_first_last": [res[0]["mean_v"], res[-1]["mean_v"]]}))


if __name__ == "__main__":
    main()
