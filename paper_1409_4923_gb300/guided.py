"""Surrogate-guided parameter scans: label, train, calibrate, screen, select, re-run.

1. Labels: the batched engine (sde_scan, one persistent launch) estimates
   (<v>, stderr) at N_label random points with N_label_paths paths each;
   half of them are drawn with an edge-dense law (see labels()).
2. Two networks of the same architecture are trained from different seeds
   on the same labels (sde_mlp_train_step).
3. Calibration on held-out labelled points (split conformal prediction with
   a normalised score): the predicted model error of a point is
   kappa (|v1 - v2| + r0), the ensemble disagreement plus the label noise
   floor r0, and kappa is the 0.999 quantile of the held-out residuals
   divided by that difficulty.
4. Screen: both networks predict every grid point (sde_mlp_forward).
5. Select: sde_guided_flags flags points whose predicted model error exceeds
   tol (0.01, the accuracy asked of the map), whose predicted Monte Carlo
   stderr at the re-run's path count exceeds se_tol (0.005), or whose
   predicted <v> changes sign against a grid neighbour.
6. Re-run: the flagged points are integrated by the engine with N_rerun
   paths under the grid point's own random counter, so a re-run value equals
   the plain Monte Carlo map's value at that point bit for bit.

The plain Monte Carlo method stays both the arbiter and the fallback.  Orchestration
only: every arithmetic step runs in libsde.so's kernels.
"""
import ctypes
import math
import time

import numpy as np

from . import engine as E
from . import surrogate as S
from . import workloads as W


def scan_stats(eng, pts, deadline_ms=0.0):
    """Run scan points through sde_scan; returns (mean_v, stderr_v) arrays."""
    res = eng.scan([dict(p, params=E.make_params(**p["params"])) for p in pts], deadline_ms)
    v = np.array([r["mean_v"] for r in res])
    se = np.array([r["stderr_v"] for r in res])
    return v, se


def features(prm, kind):
    """The seven network inputs of a parameter dict: gamma, a, omega, F, Q and
    (lambda, zeta) for the Poisson model or (b, mu) for the dichotomous one."""
    if kind == "poisson":
        return [prm["gamma"], prm["a"], prm["omega"], prm["F"], prm["Q"], prm["lambda"], prm["zeta"]]
    return [prm["gamma"], prm["a"], prm["omega"], prm["F"], prm["Q"], prm["Fb"], prm["mub"]]


def box_maps(lo, hi, log_mask):
    """Input map sending the box to [-1, 1] (log10 on masked features);
    constant features map to 0."""
    lo = np.array(lo, dtype=np.float64)
    hi = np.array(hi, dtype=np.float64)
    for c in range(7):
        if log_mask >> c & 1:
            lo[c], hi[c] = math.log10(lo[c]), math.log10(hi[c])
    width = hi - lo
    scale = np.where(width > 0, 2.0 / np.where(width > 0, width, 1.0), 0.0)
    return (lo + hi) / 2.0, scale


def train_ensemble(X, T, shift, scale, log_mask, seeds=(0, 1), steps=8000, batch=512, lr=2e-3,
                   concurrent=True):
    """Networks on the same labels, one per seed.  X, T: CUDA float32 [N, 7], [N, 2].
    With `concurrent`, each network trains from its own host thread: sde_mlp_fit
    replays its step graph on a private stream and the binding releases the
    interpreter lock during the call, so the small, latency-bound kernels of
    the networks' steps run side by side.  Each network's arithmetic is its
    own, so the trained parameters do not depend on `concurrent`."""
    import threading
    t = T.double()
    mean = t.mean(0).cpu().numpy()
    std = t.std(0).clamp_min(1e-6).cpu().numpy()
    nets = []
    for s in seeds:
        net = S.Surrogate(seed=s)
        net.set_maps(shift, scale, log_mask, mean, std)
        nets.append(net)
    hists, errors = [None] * len(nets), []

    def fit(i):
        try:
            hists[i] = nets[i].fit(X, T, steps=steps, batch=batch, lr=lr, seed=seeds[i])
        except Exception as e:        # re-raised below, in the calling thread
            errors.append(e)

    if concurrent and len(nets) > 1:
        threads = [threading.Thread(target=fit, args=(i,)) for i in range(len(nets))]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
    else:
        for i in range(len(nets)):
            fit(i)
    if errors:
        for net in nets:
            net.close()
        raise errors[0]
    return nets, hists


def predict(nets, X):
    """(v1, v2, mean log10 stderr) for CUDA inputs X [M, 7]."""
    y1 = nets[0].forward(X)
    y2 = nets[1].forward(X)
    return y1[:, 0].contiguous(), y2[:, 0].contiguous(), (0.5 * (y1[:, 1] + y2[:, 1])).contiguous()


def calibrate(nets, Xh, vh, seh, se_scale, coverage=0.999):
    """kappa of the predicted-error bound kappa (|v1 - v2| + r0) from held-out
    labels (vh, seh: their Monte Carlo estimates at the label path count).
    The residual is normalised by the difficulty |v1 - v2| + r0 rather than by
    the disagreement alone, which would make the score blow up where the two
    networks happen to agree.  Returns r0 as the bound's constant term kappa r0,
    the form sde_guided_flags takes."""
    v1, v2, lse = predict(nets, Xh)
    v1, v2 = v1.double().cpu().numpy(), v2.double().cpu().numpy()
    vm = 0.5 * (v1 + v2)
    res = np.abs(vm - vh)
    floor = 2.0 * float(np.median(seh))                    # label noise floor
    d = np.abs(v1 - v2)
    kappa = float(np.quantile(res / (d + floor), coverage))
    covered = float(np.mean(res <= kappa * (d + floor)))
    return {"kappa": kappa, "r0": kappa * floor, "floor": floor, "se_scale": se_scale, "coverage": covered,
            "rmse": float(np.sqrt(np.mean(res ** 2))), "max_res": float(res.max())}


def select(nets, v1, v2, lse, nx, ny, cal, tol, se_tol):
    """sde_guided_flags: uint8 flags (CUDA) and the flagged count."""
    import torch
    L = S._lib()
    flags = torch.zeros(nx * ny, dtype=torch.uint8, device=v1.device)
    count = torch.zeros(1, dtype=torch.int32, device=v1.device)
    rc = L.sde_guided_flags(nets[0]._net, S._ptr(v1), S._ptr(v2), S._ptr(lse), nx, ny,
                            ctypes.c_float(cal["kappa"]), ctypes.c_float(cal["r0"]),
                            ctypes.c_float(cal["se_scale"]), ctypes.c_float(tol),
                            ctypes.c_float(se_tol), S._ptr(flags), S._ptr(count))
    if rc != 0:
        raise E.SdeError(rc, L.sde_mlp_last_error(nets[0]._net).decode())
    return flags, int(count.item())


def dichot_grid_point(F, b, spp=200, transient=200, periods=2000, paths=8192, point=0):
    prm = W.dichot_point(b=float(b), F=float(F), point=int(point))
    return dict(params=prm, dt=W.period_steps(prm["omega"], spp), paths=int(paths),
                n_transient=transient * spp, n_avg=periods * spp)


class DichotGuidedScan:
    """Surrogate-guided scan of <v>(F, b) of the dichotomous model on an nx x ny
    grid (F in [-0.3, 0.3], b in [0, 2], other parameters as the 2^20-path
    workload), run stage by stage so that every stage can be timed."""

    def __init__(self, nx=1024, ny=1024, label_paths=2048, rerun_paths=8192, spp=200,
                 transient=200, periods=2000, seed=0):
        import torch
        self.nx, self.ny = nx, ny
        self.label_paths, self.rerun_paths = label_paths, rerun_paths
        self.spp, self.transient, self.periods, self.seed = spp, transient, periods, seed
        self.path_len = (transient + periods) * spp
        self.Fs, self.bs = np.linspace(-0.3, 0.3, nx), np.linspace(0.0, 2.0, ny)
        self.eng = E.Engine(0, E.make_params(**W.dichot_point()), seed=seed)
        self.torch = torch
        self.nets = None
        # launch shape of the scans from the autotuner (a probe on the grid's points)
        from . import autotune
        probe = []
        for i in range(0, nx * ny, max(1, (nx * ny) // 256)):
            pt = self.grid_point(i, rerun_paths)
            probe.append(dict(pt, params=E.make_params(**pt["params"])))
        autotune.apply_tuning(self.eng, autotune.tune_scan(0, probe, seed=seed))

    def close(self):
        self.eng.close()
        for n in self.nets or []:
            n.close()

    def grid_point(self, i, paths):
        return dichot_grid_point(self.Fs[i // self.ny], self.bs[i % self.ny], self.spp,
                                 self.transient, self.periods, paths, i)

    def labels(self, n_label, n_hold, stream=7, edge_fraction=0.5):
        """Monte Carlo labels at random points of the box (point ids above the grid's).
        A fraction edge_fraction of the points has each coordinate drawn from the
        arcsine law (density 1 / (pi sqrt(u (1 - u))) on the unit interval,
        Chebyshev-node density), which samples the box's edges several times more
        densely than the interior: a smooth regressor's error concentrates at the
        edges, where it extrapolates.  The held-out points follow the same law, so
        the calibration sees the edges as often as the labels do."""
        rng = np.random.Generator(np.random.Philox(key=self.seed, counter=[stream, 0, 0, 0]))
        n = n_label + n_hold
        u = rng.uniform(0.0, 1.0, (n, 2))
        edge = rng.uniform(0.0, 1.0, n) < edge_fraction
        u[edge] = 0.5 - 0.5 * np.cos(np.pi * u[edge])          # arcsine law
        F = -0.3 + 0.6 * u[:, 0]
        b = 2.0 * u[:, 1]
        base = self.nx * self.ny
        pts = [dichot_grid_point(f, bb, self.spp, self.transient, self.periods, self.label_paths,
                                 base + k) for k, (f, bb) in enumerate(zip(F, b))]
        v, se = scan_stats(self.eng, pts)
        X = np.array([features(p["params"], "dichot") for p in pts], dtype=np.float32)
        return X, v, se

    def train(self, X, v, se, n_label, steps=8000, batch=512):
        torch = self.torch
        T = np.stack([v, np.log10(np.maximum(se, 1e-12))], axis=1).astype(np.float32)
        lo = [0.9, 4.2, 4.9, -0.3, 5e-4, 0.0, 2.0]
        hi = [0.9, 4.2, 4.9, 0.3, 5e-4, 2.0, 2.0]
        shift, scale = box_maps(lo, hi, 0)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        self.nets, hists = train_ensemble(Xd[:n_label], Td[:n_label], shift, scale, 0, steps=steps,
                                          batch=batch)
        return Xd, hists

    def grid_inputs(self):
        torch = self.torch
        FF, BB = torch.meshgrid(torch.tensor(self.Fs, dtype=torch.float32),
                                torch.tensor(self.bs, dtype=torch.float32), indexing="ij")
        G = torch.tensor(features(W.dichot_point(), "dichot"), dtype=torch.float32).repeat(
            self.nx * self.ny, 1)
        G[:, 3] = FF.reshape(-1)
        G[:, 5] = BB.reshape(-1)
        return G.cuda()

    def screen(self):
        return predict(self.nets, self.grid_inputs())

    def rerun(self, idx):
        pts = [self.grid_point(int(i), self.rerun_paths) for i in idx]
        return scan_stats(self.eng, pts) if pts else (np.zeros(0), np.zeros(0))


def guided_dichot_scan(nx=1024, ny=1024, n_label=8192, label_paths=2048, rerun_paths=8192,
                       spp=200, transient=200, periods=2000, tol=0.01, se_tol=0.005, n_valid=2048,
                       seed=0, steps=64000, valid_stream=13, coverage=0.999, log=print, batch=512):
    """The surrogate-guided scan against plain Monte Carlo on a random sample of
    the same grid points (see the module docstring)."""
    import torch
    t_all = time.time()
    g = DichotGuidedScan(nx, ny, label_paths, rerun_paths, spp, transient, periods, seed)
    n_hold = max(2048, n_label // 8)          # the calibration's 0.999 quantile needs the sample
    t0 = time.time()
    X, v_lab, se_lab = g.labels(n_label, n_hold)
    t_label = time.time() - t0
    t0 = time.time()
    Xd, hists = g.train(X, v_lab, se_lab, n_label, steps=steps, batch=batch)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    cal = calibrate(g.nets, Xd[n_label:], v_lab[n_label:], se_lab[n_label:],
                    math.sqrt(label_paths / rerun_paths), coverage)
    log("labels %d (+%d held out) in %.1f s; training %.1f s; calibration %s" %
        (n_label, n_hold, t_label, t_train, cal))
    t0 = time.time()
    v1, v2, lse = g.screen()
    flags, nflag = select(g.nets, v1, v2, lse, nx, ny, cal, tol, se_tol)
    torch.cuda.synchronize()
    t_screen = time.time() - t0
    idx = torch.nonzero(flags).flatten().cpu().numpy()
    vmap = (0.5 * (v1 + v2)).double().cpu().numpy()
    t0 = time.time()
    v_re, _ = g.rerun(idx)
    vmap[idx] = v_re
    t_rerun = time.time() - t0
    t_guided = time.time() - t_all
    rng = np.random.Generator(np.random.Philox(key=seed, counter=[valid_stream, 0, 0, 0]))
    vidx = np.sort(rng.choice(nx * ny, size=min(n_valid, nx * ny), replace=False))
    t0 = time.time()
    v_plain, se_plain = g.rerun(vidx)
    t_valid = time.time() - t0
    err = np.abs(vmap[vidx] - v_plain)
    g.close()
    cost_plain = float(nx * ny) * rerun_paths * g.path_len
    cost_label = float(n_label + n_hold) * label_paths * g.path_len
    cost_rerun = float(len(idx)) * rerun_paths * g.path_len
    return {
        "grid": [nx, ny], "flagged": int(nflag), "flagged_fraction": nflag / float(nx * ny),
        "label_points": int(n_label + n_hold), "label_paths": int(label_paths),
        "rerun_paths": int(rerun_paths), "path_len": int(g.path_len), "train_steps": int(steps),
        "validation_points": int(len(vidx)), "validation_max_abs_err": float(err.max()),
        "validation_frac_within_0.01": float(np.mean(err <= 0.01)),
        "validation_rms_err": float(np.sqrt(np.mean(err ** 2))),
        "plain_mc_stderr_median": float(np.median(se_plain)),
        "path_steps_plain_map": cost_plain, "path_steps_labels": cost_label,
        "path_steps_reruns": cost_rerun,
        "ratio_plain_over_guided_reruns": cost_plain / max(cost_rerun, 1.0),
        "ratio_plain_over_guided_total": cost_plain / (cost_rerun + cost_label),
        "seconds": {"labels": t_label, "train": t_train, "screen_select": t_screen, "reruns": t_rerun,
                    "guided_total": t_guided, "plain_validation": t_valid},
        "points_per_s_guided": nx * ny / t_guided,
        "points_per_s_plain": len(vidx) / t_valid,
        "calibration": cal,
        "train_loss_first_last": [float(hists[0][:50].mean()), float(hists[0][-50:].mean())],
    }


def main():
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description="surrogate-guided <v>(F, b) scan of the dichotomous "
                                             "model against plain Monte Carlo")
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--labels", type=int, default=8192)
    ap.add_argument("--label-paths", type=int, default=2048)
    ap.add_argument("--rerun-paths", type=int, default=8192)
    ap.add_argument("--periods", type=int, default=2000)
    ap.add_argument("--transient", type=int, default=200)
    ap.add_argument("--valid", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=64000)
    ap.add_argument("--coverage", type=float, default=0.999)
    ap.add_argument("--batch", type=int, default=512)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    r = guided_dichot_scan(nx=a.grid, ny=a.grid, n_label=a.labels, label_paths=a.label_paths,
                           rerun_paths=a.rerun_paths, transient=a.transient, periods=a.periods,
                           n_valid=a.valid, steps=a.steps, coverage=a.coverage, batch=a.batch)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
