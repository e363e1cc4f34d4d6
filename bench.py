"""Benchmark: path-steps/s of the Monte Carlo engine on one GB300 (or N, weak scaling).

A step is one pass of the whole hot path over the workload: path init from
Philox, n_transient + n_avg predictor-corrector steps of every path with all
noise increments, the per-path Eq. 31 quotient and the FP64 ensemble
reduction (sde_run).  Default workload: 2^20 paths of the inertial washboard
with dichotomous + Gaussian noise, dt = (2 pi / 4.9) / 200, 200 + 2000 periods
(4.61e11 path-steps per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

With N > 1 (torchrun) rank r runs paths [r 2^20, (r + 1) 2^20) of one
ensemble under one seed (weak scaling), and the ranks' five FP64 sums are
added (one 40-byte all-reduce per step, the only exchange Eq. 31 needs), so
the result is <v> over N 2^20 paths; value = all ranks' path-steps / the
slowest rank's time.
"""
import argparse
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "path-steps/s (1 GB300)"
UNIT = "path-steps/s"

# Algorithmic lane operations per path-step of the inertial model with
# three-point Gaussian and one jump noise (the method's own arithmetic, counted
# from Algorithms 1-4 and the Philox definition):
#   Algorithm 1 on (x, v): 3 drift evaluations x (cos argument 1, SFU cos 1,
#   force FMA 1, damping FMA 1) = 12, state updates and trapezoid sums 10,
#   fold of x (scale, round, subtract, count) 4, window sums of v, v^2 2 -> 28
#   Algorithm 2: a quarter of one Philox4x32-10 word (10 rounds x 4 ops /
#   16 steps) 2.5, three-point selection (2 compares, 2 selects) 4, the
#   uniform of the next step from the same word (one multiply) 1       ->  7.5
#   drive a cos(w t) + F: one table value per step                      ->  1
#   Algorithm 3/4 countdown (decrement, test, add of the increment)     ->  3
#   event tail: p = 1 - exp(-mu dt) = 0.0127 x (1/4 Philox 10, log 1,
#   scale 1, floor 1, guard 3, convert 1, state 2 = 19)                 ->  0.24
ALG_OPS_PER_PATH_STEP = 39.74
# Issue slots those operations need at the least: GB300 issues the FP32 add,
# multiply and FMA of two independent paths as one packed-pair instruction,
# which covers 21 of them (the force and damping FMAs 6, the state updates
# 10, the fold's scale, subtract and count 3, the window sums 2); the other
# 18.74 take a slot each.  The ceiling is one slot per lane per clock.
ALG_SLOTS_PER_PATH_STEP = 39.74 - 21 / 2
SM_LANES = 128              # issue slots x 32 lanes per SM and clock
DEFAULT_SM_MHZ = 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {}, "fallback"


def _profile_traffic(workload):
    """DRAM bytes per launch of the step kernel from the committed ncu summary."""
    path = os.path.join(ROOT, "profiles", "point_kernel_%s.md" % workload)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+|null)", txt)
    if not m or m.group(1) == "null":
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max_over_ranks(x, device=None):
    """Max of a float over the ranks of the default process group (the slowest
    rank's time); returns x unchanged without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, world, steps, t_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return float(units_per_rank) * world * steps / t_max


def shard_range(paths_per_rank, rank):
    """Paths of rank r under weak scaling: [r P, (r + 1) P) of one ensemble
    (one seed; the path index selects the random counters), so N ranks
    integrate the first N P realisations of the same ensemble."""
    return rank * paths_per_rank, paths_per_rank


def combine_sums(sums5, device=None):
    """Eq. 31's only exchange between path ranges: the sum over ranks of the
    five FP64 sums (paths, sum vbar, sum vbar^2, sum v, sum v^2).  Without a
    process group the sums are returned as they are."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in sums5]
    t = torch.tensor([float(x) for x in sums5], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu().tolist()]


def ensemble_stats(s5, n_avg):
    """Mean, variance and standard error of Eq. 31's quotient and the time moments of v
    from the five sums (as sde_stats computes them)."""
    n = s5[0]
    mean = s5[1] / n
    var = max(0.0, (s5[2] - n * mean * mean) / (n - 1.0)) if n > 1 else 0.0
    tmean = s5[3] / (n * n_avg)
    return {"n": int(n), "mean_v": mean, "var_v": var, "stderr_v": math.sqrt(var / n),
            "tmean_v": tmean, "tvar_v": s5[4] / (n * n_avg) - tmean * tmean}


def run_engine(args):
    import torch
    import torch.distributed as dist
    from paper_1409_4923_gb300 import engine as E, workloads as W

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    spec = W.run_spec(args.workload)
    paths, dt = spec["paths"], spec["dt"]
    n_tr, n_avg = spec["n_transient"], spec["n_avg"]
    steps_per_path = n_tr + n_avg
    stream = torch.cuda.Stream()
    prm = E.make_params(**spec["params"])
    from paper_1409_4923_gb300 import autotune
    knobs = dict(autotune.DEFAULT)
    if not args.no_autotune:
        t = autotune.tune(spec["model"], prm, dt, paths, n_probe_steps=2048,
                          seed=spec["seed"], stream=stream)
        knobs = {f: t[f] for f in autotune.DEFAULT}
    first, paths = shard_range(paths, rank)
    eng = E.Engine(spec["model"], prm, seed=spec["seed"], stream=stream)
    autotune.apply_tuning(eng, knobs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB of L2

    def one_step():
        eng.run(paths, dt, n_tr, n_avg, first_path=first)

    for _ in range(args.warmup):
        one_step()
        eng.stats()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    results = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            evs[i][0].record(stream)
            one_step()
            evs[i][1].record(stream)
            results.append(combine_sums(eng.stats()["sums"], device="cuda"))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) / 1e3 for a, b in evs]
    t_total = reduce_max_over_ranks(sum(times), device="cuda")
    clocks = clk.summary()

    # end to end through the public API with host buffers: create (parameters
    # from host memory), run, read the statistics back to the host, destroy
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = E.Engine(spec["model"], E.make_params(**spec["params"]), seed=spec["seed"],
                     stream=stream)
        autotune.apply_tuning(e, knobs)
        e.run(paths, dt, n_tr, n_avg, first_path=first)
        combine_sums(e.stats()["sums"], device="cuda")
        e.close()
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = reduce_max_over_ranks(statistics.median(e2e_times), device="cuda")

    units = float(paths) * steps_per_path
    value = weak_scaling_value(units, world, args.steps, t_total)
    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", DEFAULT_SM_MHZ))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tops = n_sm * SM_LANES * sm_mhz * 1e6 / 1e12
    kernel_s = statistics.mean(times)
    achieved = ALG_SLOTS_PER_PATH_STEP * units / kernel_s / 1e12
    traffic = _profile_traffic(args.workload)
    st = ensemble_stats(results[-1], n_avg)        # all ranks' paths: one ensemble
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Philox seed %d; rank r runs paths [r 2^20, (r + 1) 2^20) of one "
                "ensemble; no dataset in the method)" % spec["seed"],
        "config": {"workload": args.workload, "paths_per_gpu": paths,
                   "steps_per_path": steps_per_path, "dt": dt, "n_transient": n_tr,
                   "n_avg": n_avg, "model": "inertial washboard",
                   "noise": "gaussian three-point + " + ("dichotomous" if "dichot" in args.workload
                                                        else "poissonian"),
                   "parallelism": "paths sharded per GPU" if world > 1 else "single GPU",
                   "l2": "flushed (256 MiB device write) between timed steps",
                   "path_arith": "fp32", "accumulators": "fp64",
                   "launch_shape": {"block_threads": knobs["block"],
                                    "grid_blocks": knobs["grid"] or "persistent",
                                    "paths_per_thread": knobs["ppt"],
                                    "steps_per_launch": knobs["steps_per_launch"] or "whole run",
                                    "chosen_by": "fixed" if args.no_autotune else "autotuner"}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops,
                     "unit": "T issue slots/s (lane)", "frac": achieved / peak_tops,
                     "traffic": traffic,
                     "peak_basis": "%d SMs x %d lanes x %.0f MHz (%s sm_max_mhz)" % (
                         n_sm, SM_LANES, sm_mhz, peak_kind),
                     "alg_slots_per_path_step": ALG_SLOTS_PER_PATH_STEP,
                     "alg_ops_per_path_step": ALG_OPS_PER_PATH_STEP},
        # host->device: the parameter record and the fold's item range;
        # device->host: five FP64 sums and the status word
        "e2e": {"value": units * world / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": E.ctypes.sizeof(E.Params) + 8,
                "d2h_bytes_per_step": 5 * 8 + 4},
        # per step: the path kernel (one launch per steps_per_launch segment) and the fold
        "gpu_launches": args.steps * (1 + (-(-steps_per_path // knobs["steps_per_launch"])
                                           if knobs["steps_per_launch"] else 1)),
        "clocks": clocks,
        "result": {"ensemble_paths": st["n"], "mean_v": st["mean_v"], "stderr_v": st["stderr_v"],
                   "tmean_v": st["tmean_v"], "tvar_v": st["tvar_v"]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, args.cpu_seconds)
    eng.close()
    if world == 1 and args.scan_valid > 0:
        line["scan"] = scan_record(args.scan_valid, local)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def scan_record(n_valid, device_index):
    """The metric's second half, measured after the timed path-steps region:
    points per second at |d<v>| <= 0.01 of the surrogate-guided 1024 x 1024
    dichotomous scan against plain Monte Carlo on the same grid, the 64 x 64
    Poissonian batched scan (one persistent launch), and that scan screened by
    networks of its own 2-D slice, validated on all of its points.

    Plain Monte Carlo is measured, not assumed: n_valid random grid points run
    through the same batched scan at the plain map's 8192 paths (their values
    are the plain map's values there, bit for bit), which gives both the
    plain method's points/s and the guided map's error on those points.  The
    plain map's full cost is extrapolated from that rate:
    t_plain_map = grid points / (n_valid / t_valid)."""
    from paper_1409_4923_gb300 import box_surrogate, guided, timing
    with ClockSampler(device_index) as clk:
        g = guided.guided_dichot_scan(n_valid=n_valid, log=lambda *a: None)
        s64 = timing.time_scan("scan_64x64", reps=2)
        gp = box_surrogate.slice_screen_64x64()
    npts = g["grid"][0] * g["grid"][1]
    t = g["seconds"]
    plain_pps = g["points_per_s_plain"]
    return {
        "guided_1024x1024": {
            "workload": "dichotomous <v>(F, b) on a 1024 x 1024 grid, 200 + 2000 periods, spp 200; "
                        "plain map at 8192 paths per point",
            "seconds": {k: round(v, 3) for k, v in t.items()},
            "points_per_s": g["points_per_s_guided"],
            "labels": {"points": g["label_points"], "paths": g["label_paths"],
                       "path_steps": g["path_steps_labels"]},
            "train": {"networks": 2, "adam_steps": g["train_steps"],
                      "heldout_rmse": g["calibration"]["rmse"],
                      "kappa": g["calibration"]["kappa"]},
            "flagged": g["flagged"], "flagged_fraction": g["flagged_fraction"],
            "path_steps_reruns": g["path_steps_reruns"],
            "path_steps_guided_total": g["path_steps_reruns"] + g["path_steps_labels"],
            "path_steps_plain_map": g["path_steps_plain_map"],
            "ratio_path_steps_plain_over_guided": g["ratio_plain_over_guided_total"],
            "validation": {"points": g["validation_points"], "paths": g["rerun_paths"],
                           "max_abs_err": g["validation_max_abs_err"],
                           "rms_err": g["validation_rms_err"],
                           "frac_within_0.01": g["validation_frac_within_0.01"],
                           "plain_stderr_median": g["plain_mc_stderr_median"]},
        },
        "plain_mc": {
            "points_per_s": plain_pps,
            "path_steps_per_s": g["validation_points"] * g["rerun_paths"] * g["path_len"] / t["plain_validation"],
            "seconds_full_map_extrapolated": npts / plain_pps,
            "formula": "grid points / (validation points / validation seconds)",
        },
        "guided_over_plain_points_per_s": g["points_per_s_guided"] / plain_pps,
        "scan_64x64": {"workload": "4096 Poisson points, 64 x 64 grid of F x log Q, paths 256..16384, "
                                   "500..3000 averaged periods, one point-kernel launch per point on "
                                   "128 side streams",
                       "seconds": s64["seconds"], "points_per_s": s64["points_per_s"],
                       "path_steps_per_s": s64["path_steps_per_s"],
                       "launch_shape": s64["launch_shape"]},
        "guided_64x64_poisson": {
            "workload": "the same 4096 points screened by networks of the (F, log Q) slice; every "
                        "point validated against the plain map",
            "labels": gp["labels"], "flagged_fraction": gp["flagged_fraction"],
            "max_abs_err": gp["max_abs_err"], "frac_within_0.01": gp["frac_within_0.01"],
            "path_steps_guided_total": gp["path_steps_guided_total"],
            "path_steps_plain_map": gp["path_steps_plain_map"],
            "ratio_path_steps_plain_over_guided": gp["ratio_plain_over_guided_total"],
            "seconds_guided_total": gp["seconds_guided_total"],
            "points_per_s_guided": 4096.0 / gp["seconds_guided_total"],
            "seconds_plain_map": gp["seconds_plain_map"],
            "points_per_s_plain": 4096.0 / gp["seconds_plain_map"]},
        "clocks": clk.summary(),
    }


def _oracle_sample(spec, paths, threads=None):
    import oracle
    prm = dict(spec["params"])
    prm["noise"] = prm.pop("noise_flags")
    p = oracle.make_params(**prm)
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.run_paths(spec["model"], p, spec["seed"], 0, paths, spec["dt"], spec["n_transient"],
                     spec["n_avg"], nthreads=cores)
    return time.perf_counter() - t0, cores


def cpu_baseline(spec, seconds):
    """The oracle as it stands, on all host cores, over a bounded sample of the
    same workload (the first paths, full horizon)."""
    steps = spec["n_transient"] + spec["n_avg"]
    cores = os.cpu_count() or 1
    probe = max(1, min(cores, 16))
    t, _ = _oracle_sample(dict(spec, n_transient=0, n_avg=max(1, steps // 20)), probe)
    rate = probe * max(1, steps // 20) / t
    paths = max(cores, int(rate * seconds / steps) // cores * cores)
    t, cores = _oracle_sample(spec, paths)
    t1, _ = _oracle_sample(spec, 2, threads=1)          # one core, as the paper's CPU baseline
    return {"value": paths * steps / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d paths, full horizon (%d steps), %.1f s wall" % (
                paths, spec["paths"], steps, t),
            "single_core_value": 2 * steps / t1}


def run_reference(args):
    """The base contract's reference arm: the FP64 CPU oracle, timed as it stands."""
    from paper_1409_4923_gb300 import workloads as W
    world, rank, _ = _dist()
    if rank != 0:
        return
    spec = W.run_spec(args.workload)
    steps = spec["n_transient"] + spec["n_avg"]
    cores = os.cpu_count() or 1
    paths = cores * 2
    for _ in range(args.warmup):
        _oracle_sample(dict(spec, n_transient=0, n_avg=steps // 50), cores)
    times = []
    for _ in range(args.steps):
        t, cores = _oracle_sample(spec, paths)
        times.append(t)
    value = paths * steps * len(times) / sum(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(times) / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Philox seed %d)" % spec["seed"], "impl": "reference",
        "config": {"workload": args.workload, "paths_per_step": paths, "steps_per_path": steps,
                   "dt": spec["dt"], "model": "inertial washboard"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d of %d paths per step, full horizon" % (paths, spec["paths"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="dichot_2p20", choices=["dichot_2p20", "poisson_1024"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default launch knobs instead of the autotuner's")
    ap.add_argument("--scan-valid", type=int, default=65536,
                    help="grid points of the plain-MC validation of the guided scan record "
                         "(0: no scan record; single GPU only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
