"""Shared helpers of the GPU parity tests (engine vs oracle on the same seeds)."""
import math

import numpy as np


def oracle_params(orc, prm):
    d = dict(prm)
    d["noise"] = d.pop("noise_flags", 0)
    return orc.make_params(**d)


def engine_run(E, torch, model, prm, seed, paths, dt, n_tr, n_avg, per_path=True, tuning=None, ppt=1):
    """Run through the C ABI; returns (stats dict, per-path numpy dict or None).
    tuning: (threads per block, grid) or None; ppt: paths per lane."""
    eng = E.Engine(model, E.make_params(**prm), seed=seed)
    try:
        if tuning:
            eng.set_tuning(*tuning)
        eng.set_paths_per_thread(ppt)
        out = None
        if per_path:
            out = {"X_f": torch.zeros(paths, dtype=torch.float64, device="cuda"),
                   "v_f": torch.zeros(paths, dtype=torch.float32, device="cuda"),
                   "vbar": torch.zeros(paths, dtype=torch.float64, device="cuda"),
                   "jP": torch.zeros(paths, dtype=torch.int32, device="cuda"),
                   "jD": torch.zeros(paths, dtype=torch.int32, device="cuda")}
        eng.run(paths, dt, n_tr, n_avg, path_out=out)
        st = eng.stats()
    finally:
        eng.close()
    if out is not None:
        out = {k: v.cpu().numpy() for k, v in out.items()}
    return st, out


def combined_tol(a, b, k=3.0):
    return k * math.sqrt(a["stderr_v"] ** 2 + b["stderr_v"] ** 2)


def events_equal(g, r, margin=1e-9):
    """Event indices equal on every path whose waiting-time quotients all keep
    `margin` away from an integer (where FP64 rounding itself could decide)."""
    keep = r["evt_margin"] > margin
    okP = np.array_equal(g["jP"][keep].astype(np.uint64), r["jP"][keep])
    okD = np.array_equal(g["jD"][keep].astype(np.uint64), r["jD"][keep])
    return okP and okD, int((~keep).sum())
