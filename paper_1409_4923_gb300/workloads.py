"""Seeded synthetic workloads (parameter sets and scan grids).

This module holds no arithmetic of the method: it only defines parameter
values, step sizes, step counts and the seeded draws of path counts and
horizons.  Both the engine's callers and the oracle's callers use it.  All
draws come from numpy's Philox bit generator with seed 0.

Workloads (the paper itself uses no dataset; these stand in for its
validation and performance runs, Secs. 6-7):
  poisson_1024    inertial washboard, Poissonian + Gaussian noise, 1024 paths,
                  dt = (2 pi / omega) / 100, 100 transient + 400 averaged periods
  dichot_2p20     the same equation with dichotomous noise (b = 0.5, mu = 2)
                  and Q = 5e-4, 2^20 paths, dt = (2 pi / omega) / 200,
                  200 + 2000 periods
  scan_64x64      4096 Poisson-model points: F in [-0.3, 0.3] x log-uniform Q in
                  [1e-4, 1e-1]; paths log-uniform in [256, 16384]; averaged
                  periods uniform in [500, 3000] after 100 transient periods
  surrogate_box   2^17 points uniform in the 7-D box of (gamma, a, omega, F,
                  log10 Q, lambda, zeta), 4096 paths, 100 + 400 periods
  guided_grid     1024 x 1024 grid of F in [-0.3, 0.3] x b in [0, 2] of the
                  dichotomous model, other values as dichot_2p20
"""
import math

import numpy as np

INERTIAL_WASHBOARD = 0
NOISE_GAUSS, NOISE_POISSON, NOISE_DICHOT = 1, 2, 4

BASE = dict(gamma=0.9, a=4.2, omega=4.9, F=0.1, V0=1.0,
            x0_lo=0.0, x0_hi=1.0, v0_lo=-2.0, v0_hi=2.0)


def poisson_point(**over):
    d = dict(BASE, Q=0.001, zeta=0.1, noise_flags=NOISE_GAUSS | NOISE_POISSON)
    d["lambda"] = 1.0
    d.update(over)
    return d


def dichot_point(b=0.5, mu=2.0, **over):
    d = dict(BASE, Q=0.0005, Fa=b, Fb=b, mua=mu, mub=mu, noise_flags=NOISE_GAUSS | NOISE_DICHOT)
    d.update(over)
    return d


def period_steps(omega, spp):
    """Step size for `spp` steps per drive period 2 pi / omega."""
    return (2.0 * math.pi / omega) / spp


def run_spec(name):
    """Single-point workloads: dict(model, params, dt, paths, n_transient, n_avg, seed)."""
    if name == "poisson_1024":
        spp = 100
        return dict(model=INERTIAL_WASHBOARD, params=poisson_point(), dt=period_steps(4.9, spp),
                    paths=1024, n_transient=100 * spp, n_avg=400 * spp, seed=0)
    if name == "dichot_2p20":
        spp = 200
        return dict(model=INERTIAL_WASHBOARD, params=dichot_point(), dt=period_steps(4.9, spp),
                    paths=1 << 20, n_transient=200 * spp, n_avg=2000 * spp, seed=0)
    raise KeyError(name)


def _rng(stream):
    return np.random.Generator(np.random.Philox(key=0, counter=[stream, 0, 0, 0]))


def scan_64x64(nF=64, nQ=64, spp=100, transient_periods=100):
    """Poisson-model scan points (list of dicts, point ids 0..nF*nQ-1)."""
    rng = _rng(1)
    F = np.linspace(-0.3, 0.3, nF)
    Q = np.logspace(-4, -1, nQ)
    n = nF * nQ
    paths = np.exp(rng.uniform(math.log(256), math.log(16384), n)).round().astype(np.int64)
    periods = rng.uniform(500, 3000, n).round().astype(np.int64)
    dt = period_steps(4.9, spp)
    pts = []
    for i in range(n):
        iF, iQ = divmod(i, nQ)
        prm = poisson_point(F=float(F[iF]), Q=float(Q[iQ]), point=i)
        pts.append(dict(params=prm, dt=dt, paths=int(paths[i]), n_transient=transient_periods * spp,
                        n_avg=int(periods[i]) * spp, F=float(F[iF]), Q=float(Q[iQ])))
    return pts


SURROGATE_BOX = dict(gamma=(0.5, 1.5), a=(2.0, 6.0), omega=(3.0, 7.0), F=(-0.3, 0.3),
                     log10Q=(-4.0, -1.0), **{"lambda": (0.1, 5.0)}, zeta=(0.01, 0.5))
SURROGATE_KEYS = ("gamma", "a", "omega", "F", "log10Q", "lambda", "zeta")


def surrogate_box_points(n=1 << 17, spp=100, transient_periods=100, avg_periods=400, paths=4096,
                         stream=2, edge_fraction=0.0):
    """Draws in the 7-D box; returns (X[n,7] box coordinates with log10 Q, list of
    scan points).  A fraction edge_fraction of the points has each coordinate
    drawn from the arcsine law (density 1 / (pi sqrt(u (1 - u))) on the unit
    interval), which samples the box's faces more densely; the rest is uniform."""
    rng = _rng(stream)
    U = rng.uniform(0.0, 1.0, (n, len(SURROGATE_KEYS)))
    if edge_fraction > 0.0:
        edge = rng.uniform(0.0, 1.0, n) < edge_fraction
        U[edge] = 0.5 - 0.5 * np.cos(np.pi * U[edge])
    lo = np.array([SURROGATE_BOX[k][0] for k in SURROGATE_KEYS])
    hi = np.array([SURROGATE_BOX[k][1] for k in SURROGATE_KEYS])
    X = lo + (hi - lo) * U
    pts = []
    for i in range(n):
        g, a, w, F, lq, lam, zeta = X[i]
        prm = poisson_point(gamma=g, a=a, omega=w, F=F, Q=10.0 ** lq, zeta=zeta, point=i)
        prm["lambda"] = lam
        pts.append(dict(params=prm, dt=period_steps(w, spp), paths=paths,
                        n_transient=transient_periods * spp, n_avg=avg_periods * spp))
    return X, pts


def guided_grid(nF=1024, nb=1024):
    """(F values, b values) of the dichotomous guided-scan grid."""
    return np.linspace(-0.3, 0.3, nF), np.linspace(0.0, 2.0, nb)
