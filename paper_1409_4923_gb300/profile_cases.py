"""Small, self-contained launches for profiling the engine's kernels.

  python -m paper_1409_4923_gb300.profile_cases point dichot_2p20 --paths 1048576 --steps 800 [--ppt 2]
  python -m paper_1409_4923_gb300.profile_cases mlp --rows 1048576 --path 1
  python -m paper_1409_4923_gb300.profile_cases scan --points 256
  python -m paper_1409_4923_gb300.profile_cases scan_dichot --points 64 --paths 16384 --steps 4096
  python -m paper_1409_4923_gb300.profile_cases fit --rows 16384 --steps 200

Each case runs its launch twice (a warm-up and the one to capture) and
prints a checksum, so `ncu --clock-control none -s 1 -c 1 -k <kernel>` captures a warm launch.
"""
import argparse
import sys


def main():
    import numpy as np
    import torch
    from . import engine as E, workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["point", "mlp", "scan", "scan_dichot", "fit"])
    ap.add_argument("workload", nargs="?", default="dichot_2p20")
    ap.add_argument("--paths", type=int, default=1 << 20)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--rows", type=int, default=1 << 20)
    ap.add_argument("--points", type=int, default=256)
    ap.add_argument("--path", type=int, default=1, help="mlp: 1 tcgen05, 0 mma.sync")
    ap.add_argument("--ppt", type=int, default=1, help="point: paths per lane (1 or 2)")
    ap.add_argument("--batch", type=int, default=512, help="fit: minibatch rows")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.case == "point":
        spec = W.run_spec(a.workload)
        eng = E.Engine(spec["model"], E.make_params(**spec["params"]), seed=spec["seed"])
        eng.set_paths_per_thread(a.ppt)
        for _ in range(2):
            eng.run(a.paths, spec["dt"], 0, a.steps)
            print("mean_v", eng.stats()["mean_v"])
        eng.close()
    elif a.case == "mlp":
        from . import surrogate as S
        rng = np.random.default_rng(0)
        x = torch.from_numpy(rng.uniform(0.5, 1.5, (a.rows, 7)).astype(np.float32)).cuda()
        net = S.Surrogate(0)
        net.set_tensor_path(a.path)
        for _ in range(2):
            y = net.forward(x)
            net.sync()
            print("checksum", float(y.double().sum()))
        net.close()
    elif a.case == "fit":
        from . import surrogate as S
        rng = np.random.default_rng(0)
        x = torch.from_numpy(rng.uniform(0.5, 1.5, (a.rows, 7)).astype(np.float32)).cuda()
        t = torch.from_numpy(rng.normal(0.0, 1.0, (a.rows, 2)).astype(np.float32)).cuda()
        net = S.Surrogate(0)
        for _ in range(2):
            hist = net.fit(x, t, steps=a.steps, batch=a.batch)
            print("loss first/last", float(hist[0]), float(hist[-1]))
        net.close()
    elif a.case == "scan_dichot":
        # dichotomous points of equal size through the persistent scan kernel
        # (two paths per lane), 128-thread blocks
        pts = [dict(params=E.make_params(**W.dichot_point(b=0.5, F=0.1, point=i)),
                    dt=W.period_steps(4.9, 200), paths=a.paths, n_transient=0, n_avg=a.steps)
               for i in range(a.points)]
        eng = E.Engine(0, pts[0]["params"], seed=0)
        eng.set_tuning(128, 0)
        eng.set_scan_mode(1)
        for _ in range(2):
            print("mean_v[0]", eng.scan(pts)[0]["mean_v"])
        eng.close()
    else:
        pts = W.scan_64x64()[:a.points]
        eng = E.Engine(0, E.make_params(**pts[0]["params"]), seed=0)
        arg = [dict(p, params=E.make_params(**p["params"]), n_avg=min(p["n_avg"], a.steps)) for p in pts]
        for _ in range(2):
            res = eng.scan(arg)
            print("mean_v[0]", res[0]["mean_v"])
        eng.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
