"""Plain FP64 CPU oracle of the Brownian-motor Monte Carlo method (ctypes binding).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import it; the engine package never does.
It shares no code with the CUDA engine.  Everything numeric lives in
sde_oracle.c (Algorithms 1-4 of the paper, step by step, in double
precision); this module only marshals arguments.

Parity status per function (details in the pins under tests/):
  philox4x32_10  pinned (Triton's independent Philox in interpreter mode)
  noise_sequence pinned (exact three-point moments, Binomial Poisson counts,
                 amplitude law, dichotomous correlation and occupation)
  run_paths      pinned for the free, linear (OU), overdamped washboard
                 (Stratonovich), piecewise-linear (Eqs. 21-23) and inertial
                 free/equipartition/driven-linear cases, and for the inertial
                 driven washboard with the noise off (second-order convergence
                 to SciPy's DOP853); with noise that model has no closed form:
                 parity unpinned beyond those pins.
"""
import ctypes
import os

import numpy as np

from . import build as _build

INERTIAL_WASHBOARD, OVERDAMPED_WASHBOARD, OVERDAMPED_PWL, OVERDAMPED_LINEAR = 0, 1, 2, 3
GAUSS, POISSON, DICHOT, GAUSS_NORMAL, POIS_COMPENSATED, DICHOT_IN_DRIFT = 1, 2, 4, 8, 16, 32


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "gamma", "a", "omega", "F", "Q", "lambda_", "zeta", "Fa", "Fb", "mua", "mub",
        "V0", "x0_lo", "x0_hi", "v0_lo", "v0_hi")] + [
        ("noise", ctypes.c_uint32), ("point", ctypes.c_uint32)]


PATH_DTYPE = np.dtype([
    ("X_f", "f8"), ("v_f", "f8"), ("X_i", "f8"), ("vbar", "f8"), ("sum_v", "f8"),
    ("sum_v2", "f8"), ("kink_min", "f8"), ("evt_margin", "f8"), ("jP", "u8"),
    ("jD", "u8"), ("d", "i4"), ("pad", "i4")])

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.orc_philox_many.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.c_void_p]
        L.orc_local_error.argtypes = [ctypes.c_int, ctypes.POINTER(Params), ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.orc_local_error.restype = ctypes.c_int
        L.orc_run_paths.argtypes = [ctypes.c_int, ctypes.POINTER(Params), ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.c_void_p]
        L.orc_run_paths.restype = ctypes.c_int
        L.orc_stats.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.POINTER(ctypes.c_double)]
        L.orc_noise_sequence.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Params),
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_void_p]
        L.orc_noise_sequence.restype = ctypes.c_int
        L.orc_stream_words.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_uint32)]
        _lib = L
    return _lib


def make_params(**kw) -> Params:
    """Build a Params record; unspecified fields are 0 except V0 = 1."""
    p = Params()
    p.V0 = 1.0
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if k == "noise":
            p.noise = int(v)
        elif k == "point":
            p.point = int(v)
        else:
            setattr(p, k, float(v))
    return p


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def philox_many(ctr, key):
    """Philox4x32-10 of an (n, 4) uint32 array of counters under one key -> (n, 4) words."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros_like(ctr)
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    lib().orc_philox_many(ctr.ctypes.data, ctr.shape[0], k, out.ctypes.data)
    return out


def local_error(model, params: Params, seed, path0, npaths, dt, n_steps, nthreads=None):
    """Sec. 4's chi over npaths paths x n_steps steps: dict of rms and max of
    chi_x (x units) and chi_v (inertial model)."""
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    o = (ctypes.c_double * 4)()
    rc = lib().orc_local_error(model, ctypes.byref(params), seed, path0, npaths, dt, n_steps,
                               nthreads, o)
    if rc != 0:
        raise ValueError("orc_local_error rejected its arguments")
    n = float(npaths) * float(n_steps)
    return {"rms_x": (o[0] / n) ** 0.5, "rms_v": (o[1] / n) ** 0.5, "max_x": o[2], "max_v": o[3]}


def stream_words(seed, tag, point, path, idx):
    o = (ctypes.c_uint32 * 4)()
    lib().orc_stream_words(seed, tag, point, path, idx, o)
    return [int(x) for x in o]


def run_paths(model, params: Params, seed, path0, npaths, dt, n_transient, n_avg, nthreads=None):
    """Integrate paths path0..path0+npaths-1; returns a structured array (PATH_DTYPE)."""
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    out = np.zeros(int(npaths), dtype=PATH_DTYPE)
    rc = lib().orc_run_paths(int(model), ctypes.byref(params), int(seed), int(path0),
                             int(npaths), float(dt), int(n_transient), int(n_avg),
                             int(nthreads), out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_run_paths rejected its arguments")
    return out


def stats(out, n_avg):
    """Eq. 31 ensemble statistics: dict(n, mean_v, var_v, stderr_v, tmean_v, tvar_v, s, s2)."""
    res = (ctypes.c_double * 8)()
    out = np.ascontiguousarray(out)
    lib().orc_stats(out.ctypes.data, len(out), int(n_avg), res)
    keys = ("n", "mean_v", "var_v", "stderr_v", "tmean_v", "tvar_v", "sum_vbar", "sum_vbar2")
    return dict(zip(keys, [float(x) for x in res]))


def noise_sequence(kind, model, params: Params, seed, path, dt, n):
    """kind 1: Gaussian increments, 2: Poisson increments, 3: dichotomous values."""
    out = np.zeros(int(n), dtype=np.float64)
    rc = lib().orc_noise_sequence(int(kind), int(model), ctypes.byref(params), int(seed),
                                  int(path), float(dt), int(n), out.ctypes.data)
    if rc != 0:
        raise ValueError("orc_noise_sequence rejected its arguments")
    return out
