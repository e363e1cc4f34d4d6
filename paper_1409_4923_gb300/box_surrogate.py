"""The surrogate of the Poisson model over its 7-D parameter box, end to end.

  python -m paper_1409_4923_gb300.box_surrogate            # 2^17 labels, 2^20-point inference

1. Labels: points drawn uniformly in the box (gamma, a, omega, F, log10 Q,
   lambda, zeta; workloads.SURROGATE_BOX) are integrated by the batched engine
   in one persistent scan (4096 paths, 100 + 400 drive periods, 100 steps per
   period), giving (<v>, stderr) per point; a further eighth of the points is
   held out.
2. Training: two networks from different seeds on (<v>, log10 stderr), with
   the engine's own forward / backward / Adam kernels (surrogate.Surrogate).
3. Held-out accuracy of <v> and log10 stderr.
4. Inference: the two networks over 2^20 fresh points of the box, timed.

Orchestration only: every arithmetic step runs in libsde.so's kernels.
"""
import json
import time

import numpy as np

from . import autotune
from . import engine as E
from . import guided
from . import workloads as W

LOG_MASK = 1 << 4          # Q enters the network through log10


def box_bounds():
    keys = ("gamma", "a", "omega", "F")
    lo = [W.SURROGATE_BOX[k][0] for k in keys] + [10.0 ** W.SURROGATE_BOX["log10Q"][0]] + \
         [W.SURROGATE_BOX["lambda"][0], W.SURROGATE_BOX["zeta"][0]]
    hi = [W.SURROGATE_BOX[k][1] for k in keys] + [10.0 ** W.SURROGATE_BOX["log10Q"][1]] + \
         [W.SURROGATE_BOX["lambda"][1], W.SURROGATE_BOX["zeta"][1]]
    return lo, hi


def raw_inputs(X):
    """Network inputs from box draws: the box holds log10 Q, the network Q."""
    Xr = np.array(X, dtype=np.float64)
    Xr[:, 4] = 10.0 ** Xr[:, 4]
    return Xr.astype(np.float32)


def run(n_label=1 << 17, paths=4096, steps=32000, batch=1024, n_infer=1 << 20, seed=0, log=print):
    import torch
    n_hold = n_label // 8
    X, pts = W.surrogate_box_points(n=n_label + n_hold, paths=paths)
    eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=seed)
    try:
        scan_pts = [dict(p, params=E.make_params(**p["params"])) for p in pts]
        autotune.apply_tuning(eng, autotune.tune_scan(0, scan_pts[::64], seed=seed))
        torch.cuda.synchronize()
        t0 = time.time()
        res = eng.scan(scan_pts)
        t_label = time.time() - t0
    finally:
        eng.close()
    v = np.array([r["mean_v"] for r in res])
    se = np.array([r["stderr_v"] for r in res])
    path_steps = float(sum(p["paths"] * (p["n_transient"] + p["n_avg"]) for p in pts))
    log("labels: %d points, %.3g path-steps in %.1f s" % (len(pts), path_steps, t_label))

    T = np.stack([v, np.log10(np.maximum(se, 1e-12))], axis=1).astype(np.float32)
    Xd = torch.from_numpy(raw_inputs(X)).cuda()
    Td = torch.from_numpy(T).cuda()
    shift, scale = guided.box_maps(*box_bounds(), LOG_MASK)
    t0 = time.time()
    nets, hists = guided.train_ensemble(Xd[:n_label], Td[:n_label], shift, scale, LOG_MASK, steps=steps,
                                        batch=batch)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    try:
        v1, v2, lse = guided.predict(nets, Xd[n_label:])
        vm = (0.5 * (v1 + v2)).double().cpu().numpy()
        res_v = vm - v[n_label:]
        res_l = lse.double().cpu().numpy() - T[n_label:, 1]
        # inference over fresh points of the box, timed on the device
        rng = np.random.Generator(np.random.Philox(key=seed, counter=[29, 0, 0, 0]))
        keys = W.SURROGATE_KEYS
        Xi = np.stack([rng.uniform(*W.SURROGATE_BOX[k], n_infer) for k in keys], axis=1)
        Xi = torch.from_numpy(raw_inputs(Xi)).cuda()
        nets[0].forward(Xi)
        nets[0].sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for net in nets:
            net.forward(Xi)
        ev1.record()
        for net in nets:
            net.sync()
        t_infer = ev0.elapsed_time(ev1) / 1e3 / len(nets)
    finally:
        for net in nets:
            net.close()
    return {
        "labels": len(pts), "label_paths": paths, "label_path_steps": path_steps,
        "label_seconds": t_label, "label_points_per_s": len(pts) / t_label,
        "label_path_steps_per_s": path_steps / t_label,
        "train_steps": steps, "train_seconds": t_train,
        "heldout": int(n_hold), "heldout_v_rmse": float(np.sqrt(np.mean(res_v ** 2))),
        "heldout_v_mae": float(np.mean(np.abs(res_v))),
        "heldout_v_q99": float(np.quantile(np.abs(res_v), 0.99)),
        "label_v_std": float(v[n_label:].std()), "label_stderr_median": float(np.median(se)),
        "heldout_log10_stderr_rmse": float(np.sqrt(np.mean(res_l ** 2))),
        "train_loss_first_last": [float(hists[0][:100].mean()), float(hists[0][-100:].mean())],
        "inference_points": int(n_infer), "inference_seconds_per_network": t_infer,
        "inference_points_per_s": n_infer / t_infer,
    }


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="surrogate of the Poisson model over its 7-D box")
    ap.add_argument("--labels", type=int, default=1 << 17)
    ap.add_argument("--paths", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=32000)
    ap.add_argument("--infer", type=int, default=1 << 20)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    print(json.dumps(run(n_label=a.labels, paths=a.paths, steps=a.steps, n_infer=a.infer)))


if __name__ == "__main__":
    main()
