"""The surrogate of the Poisson model over its 7-D parameter box, end to end.

  python -m paper_1409_4923_gb300.box_surrogate            # 2^17 labels, 2^20-point inference

1. Labels: points of the box (gamma, a, omega, F, log10 Q, lambda, zeta;
   workloads.SURROGATE_BOX), half uniform and half edge-dense, are integrated
   by the batched engine in one persistent scan (4096 paths, 100 + 400 drive
   periods, 100 steps per period), giving (<v>, stderr) per point; a further
   eighth of the points (the same mixture) is held out.
2. Training: two networks from different seeds on (<v>, log10 stderr), with
   the engine's own forward / backward / Adam kernels (surrogate.Surrogate);
   Q, lambda and zeta enter through log10.
3. Held-out accuracy of <v> and log10 stderr, and the calibration of the
   predicted model error (guided.calibrate).
4. Inference: the two networks over 2^20 fresh points of the box, timed.
5. Guided screen of the 64 x 64 Poisson scan (workloads.scan_64x64): the
   networks predict every grid point, sde_guided_flags selects the points to
   re-run, the engine re-runs them with the points' own path counts, horizons
   and random counters, and the guided map is compared with the plain map of
   all 4096 points.

Orchestration only: every arithmetic step runs in libsde.so's kernels.
"""
import json
import time

import numpy as np

from . import autotune
from . import engine as E
from . import guided
from . import workloads as W

LOG_MASK = (1 << 4) | (1 << 5) | (1 << 6)    # Q, lambda and zeta enter through log10


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


def screen_scan_64x64(nets, cal, label_paths, label_periods=400, tol=0.01, se_tol=0.005, seed=0,
                      plain=None):
    """Guided screen of the 64 x 64 Poisson scan with the box networks (step 5).
    The predicted Monte Carlo stderr of a point is the networks' label stderr
    rescaled to the point's own path count N and averaged periods T
    (stderr ~ 1 / sqrt(N T) for Eq. 31's quotient).  plain: the plain map's
    (<v>, stderr) of all points, computed here when not given."""
    import torch
    from . import surrogate as S
    pts = W.scan_64x64()
    nF = nQ = 64
    X = np.array([guided.features(p["params"], "poisson") for p in pts], dtype=np.float32)
    v1, v2, lse = guided.predict(nets, torch.from_numpy(X).cuda())
    spp = 100                                   # steps per drive period of the scan
    shift = np.array([0.5 * np.log10(label_paths * label_periods / (p["paths"] * p["n_avg"] / spp))
                      for p in pts], dtype=np.float32)
    lse_pt = (lse + torch.from_numpy(shift).cuda()).contiguous()
    flags, nflag = guided.select(nets, v1, v2, lse_pt, nF, nQ, dict(cal, se_scale=1.0), tol, se_tol)
    idx = torch.nonzero(flags).flatten().cpu().numpy()
    vmap = (0.5 * (v1 + v2)).double().cpu().numpy()
    eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=seed)
    try:
        torch.cuda.synchronize()
        t0 = time.time()
        if len(idx):
            v_re, _ = guided.scan_stats(eng, [pts[i] for i in idx])
            vmap[idx] = v_re
        t_rerun = time.time() - t0
        if plain is None:
            t0 = time.time()
            plain = guided.scan_stats(eng, pts)
            t_plain = time.time() - t0
        else:
            t_plain = None
    finally:
        eng.close()
    v_plain, se_plain = plain
    err = np.abs(vmap - v_plain)
    cost = np.array([p["paths"] * (p["n_transient"] + p["n_avg"]) for p in pts], dtype=np.float64)
    return {"grid": [nF, nQ], "flagged": int(nflag), "flagged_fraction": nflag / float(nF * nQ),
            "max_abs_err": float(err.max()), "frac_within_0.01": float(np.mean(err <= tol)),
            "rms_err": float(np.sqrt(np.mean(err ** 2))),
            "path_steps_reruns": float(cost[idx].sum()), "path_steps_plain_map": float(cost.sum()),
            "ratio_plain_over_reruns": float(cost.sum() / max(cost[idx].sum(), 1.0)),
            "seconds_reruns": t_rerun, "seconds_plain_map": t_plain,
            "plain_stderr_median": float(np.median(se_plain))}


def slice_screen_64x64(n_label=1024, n_hold=256, label_paths=4096, label_periods=400, steps=10000,
                       batch=512, tol=0.01, se_tol=0.005, seed=0, coverage=0.999, plain=None):
    """Guided screen of the 64 x 64 Poisson scan with networks of its own 2-D
    slice (F, log10 Q; the other five parameters as the scan's), the
    construction of the dichotomous guided scan: labels half uniform and half
    edge-dense on the slice (point ids above the grid's), two networks,
    split-conformal calibration on held-out labels, screen, re-run of the
    flagged points with their own path counts, horizons and random counters,
    and comparison with the plain map of all 4096 points.  Path-steps are
    counted for labels and re-runs together."""
    import torch
    pts = W.scan_64x64()
    n = n_label + n_hold
    rng = np.random.Generator(np.random.Philox(key=seed, counter=[31, 0, 0, 0]))
    u = rng.uniform(0.0, 1.0, (n, 2))
    edge = rng.uniform(0.0, 1.0, n) < 0.5
    u[edge] = 0.5 - 0.5 * np.cos(np.pi * u[edge])
    F = -0.3 + 0.6 * u[:, 0]
    Q = 10.0 ** (-4.0 + 3.0 * u[:, 1])
    spp = 100
    lab = [dict(params=W.poisson_point(F=float(f), Q=float(q), point=len(pts) + k),
                dt=pts[0]["dt"], paths=label_paths, n_transient=100 * spp, n_avg=label_periods * spp)
           for k, (f, q) in enumerate(zip(F, Q))]
    eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=seed)
    try:
        torch.cuda.synchronize()
        t0 = time.time()
        v, se = guided.scan_stats(eng, lab)
        t_label = time.time() - t0
        X = np.array([guided.features(p["params"], "poisson") for p in lab], dtype=np.float32)
        T = np.stack([v, np.log10(np.maximum(se, 1e-12))], axis=1).astype(np.float32)
        base = pts[0]["params"]
        lo = [base["gamma"], base["a"], base["omega"], -0.3, 1e-4, base["lambda"], base["zeta"]]
        hi = [base["gamma"], base["a"], base["omega"], 0.3, 1e-1, base["lambda"], base["zeta"]]
        shift, scale = guided.box_maps(lo, hi, 1 << 4)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        t0 = time.time()
        nets, _ = guided.train_ensemble(Xd[:n_label], Td[:n_label], shift, scale, 1 << 4, steps=steps,
                                        batch=batch)
        torch.cuda.synchronize()
        t_train = time.time() - t0
        try:
            cal = guided.calibrate(nets, Xd[n_label:], v[n_label:], se[n_label:], 1.0, coverage)
            scr = screen_scan_64x64(nets, cal, label_paths, label_periods, tol, se_tol, seed, plain)
        finally:
            for net in nets:
                net.close()
    finally:
        eng.close()
    cost_label = float(n) * label_paths * (100 + label_periods) * spp
    total = cost_label + scr["path_steps_reruns"]
    scr.update({"labels": n, "label_paths": label_paths, "label_seconds": t_label,
                "train_seconds": t_train, "calibration": cal, "path_steps_labels": cost_label,
                "path_steps_guided_total": total,
                "ratio_plain_over_guided_total": scr["path_steps_plain_map"] / total,
                "seconds_guided_total": t_label + t_train + scr["seconds_reruns"]})
    return scr


def run(n_label=1 << 17, paths=4096, steps=256000, batch=1024, n_infer=1 << 20, seed=0, log=print,
        edge_fraction=0.5, screen=True):
    import torch
    n_hold = n_label // 8
    X, pts = W.surrogate_box_points(n=n_label + n_hold, paths=paths, edge_fraction=edge_fraction)
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
        cal = guided.calibrate(nets, Xd[n_label:], v[n_label:], se[n_label:], 1.0)
        scr = screen_scan_64x64(nets, cal, paths, seed=seed) if screen else None
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
        "calibration": cal, "screen_scan_64x64": scr,
    }


def main():
    import argparse
    import torch
    ap = argparse.ArgumentParser(description="surrogate of the Poisson model over its 7-D box")
    ap.add_argument("--labels", type=int, default=1 << 17)
    ap.add_argument("--paths", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=256000)
    ap.add_argument("--infer", type=int, default=1 << 20)
    ap.add_argument("--slice", action="store_true",
                    help="only the 64 x 64 scan's guided screen with networks of its 2-D slice")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.slice:
        print(json.dumps(slice_screen_64x64()))
        return
    print(json.dumps(run(n_label=a.labels, paths=a.paths, steps=a.steps, n_infer=a.infer)))


if __name__ == "__main__":
    main()
