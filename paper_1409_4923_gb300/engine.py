"""ctypes binding of the engine's C ABI (include/sde.h).

Argument marshalling only: every step of the Monte Carlo path runs in the CUDA
kernels of libsde.so.  PyTorch supplies device buffers (per-path outputs) and
the CUDA stream.  There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.
"""
import ctypes
import os
import struct

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsde.so")

INERTIAL_WASHBOARD, OVERDAMPED_WASHBOARD, OVERDAMPED_PWL = 0, 1, 2
NOISE_GAUSS, NOISE_POISSON, NOISE_DICHOT, GAUSS_NORMAL, POIS_COMPENSATED = 1, 2, 4, 8, 16

SDE_OK, SDE_EINVAL, SDE_ECUDA, SDE_ENOMEM, SDE_ETIMEDOUT, SDE_ESTATE = 0, -1, -2, -3, -4, -5
_CODES = {-1: "EINVAL", -2: "ECUDA", -3: "ENOMEM", -4: "ETIMEDOUT", -5: "ESTATE"}


class SdeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_CODES.get(code, code), msg))
        self.code = code


class SdeTimeout(SdeError):
    pass


class Params(ctypes.Structure):
    """Mirror of sde_params."""
    _fields_ = [(n, ctypes.c_double) for n in (
        "gamma", "a", "omega", "F", "Q", "lambda_", "zeta", "Fa", "Fb", "mua", "mub", "V0",
        "x0_lo", "x0_hi", "v0_lo", "v0_hi")] + [
        ("noise_flags", ctypes.c_uint32), ("point", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    """Mirror of sde_stats_t."""
    _fields_ = [("n", ctypes.c_uint64), ("mean_v", ctypes.c_double), ("var_v", ctypes.c_double),
                ("stderr_v", ctypes.c_double), ("tmean_v", ctypes.c_double),
                ("tvar_v", ctypes.c_double), ("sums", ctypes.c_double * 5),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {"n": int(self.n), "mean_v": self.mean_v, "var_v": self.var_v,
                "stderr_v": self.stderr_v, "tmean_v": self.tmean_v, "tvar_v": self.tvar_v,
                "sums": list(self.sums), "status": int(self.status)}


class PathOut(ctypes.Structure):
    _fields_ = [("X_f", ctypes.c_void_p), ("v_f", ctypes.c_void_p), ("vbar", ctypes.c_void_p),
                ("jP", ctypes.c_void_p), ("jD", ctypes.c_void_p)]


class ScanPoint(ctypes.Structure):
    _fields_ = [("p", Params), ("dt", ctypes.c_double), ("paths", ctypes.c_uint64),
                ("n_transient", ctypes.c_uint64), ("n_avg", ctypes.c_uint64)]


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libsde.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsde.so not built (run __graft_entry__.build()); the engine has no "
                          "CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "sde_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(Params),
                                      ctypes.c_uint64, _P]),
        "sde_set_params": (ctypes.c_int, [_P, ctypes.POINTER(Params)]),
        "sde_run": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_uint64]),
        "sde_run_paths": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.POINTER(PathOut)]),
        "sde_run_range": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(PathOut)]),
        "sde_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
        "sde_scan": (ctypes.c_int, [_P, ctypes.POINTER(ScanPoint), ctypes.c_uint32,
                                    ctypes.POINTER(Stats), ctypes.c_double]),
        "sde_scan_resume": (ctypes.c_int, [_P, ctypes.POINTER(Stats), ctypes.c_double]),
        "sde_scan_device": (ctypes.c_int, [_P, ctypes.POINTER(ScanPoint), ctypes.c_uint32, _P]),
        "sde_begin": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint64]),
        "sde_advance": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(PathOut),
                                       ctypes.POINTER(ctypes.c_uint64)]),
        "sde_checkpoint_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
        "sde_checkpoint": (ctypes.c_int, [_P, _P, ctypes.c_uint64]),
        "sde_restore": (ctypes.c_int, [_P, _P, ctypes.c_uint64]),
        "sde_local_error": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_double)]),
        "sde_reduce_f64": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
        "sde_philox_words": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_uint64, _P]),
        "sde_set_tuning": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
        "sde_set_paths_per_thread": (ctypes.c_int, [_P, ctypes.c_int]),
        "sde_set_steps_per_launch": (ctypes.c_int, [_P, ctypes.c_uint64]),
        "sde_set_scan_mode": (ctypes.c_int, [_P, ctypes.c_int]),
        "sde_occupancy": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
        "sde_run_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Params), ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.c_uint64, _P, _P, _P]),
        "sde_destroy": (None, [_P]),
        "sde_last_error": (ctypes.c_char_p, [_P]),
        "sde_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def make_params(**kw) -> Params:
    """sde_params from keywords (lambda may be spelled `lambda`); V0 defaults to 1."""
    p = Params()
    p.V0 = 1.0
    for k, v in kw.items():
        if k == "lambda":
            k = "lambda_"
        if k in ("noise", "noise_flags"):
            p.noise_flags = int(v)
        elif k == "point":
            p.point = int(v)
        else:
            setattr(p, k, float(v))
    return p


def _check(ctx, rc):
    if rc != SDE_OK:
        msg = lib().sde_last_error(ctx).decode()
        if rc == SDE_ETIMEDOUT:
            raise SdeTimeout(rc, msg)
        raise SdeError(rc, msg)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Engine:
    """One engine context: a model, its parameters, a seed and a CUDA stream."""

    def __init__(self, model, params: Params, seed=0, stream=None):
        L = lib()
        self._ctx = _P()
        self._params = params
        rc = L.sde_create(ctypes.byref(self._ctx), int(model), ctypes.byref(params),
                          int(seed), _stream_handle(stream))
        if rc != SDE_OK:
            raise SdeError(rc, L.sde_last_error(None).decode())
        self.model = model
        self._seg_paths = 0        # paths of the segmented run (begin / restore)
        self._scan_n = 0           # points of the last scan (scan_resume)

    def close(self):
        if self._ctx:
            lib().sde_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params: Params):
        _check(self._ctx, lib().sde_set_params(self._ctx, ctypes.byref(params)))
        self._params = params

    def set_tuning(self, block_threads=128, grid_blocks=0):
        _check(self._ctx, lib().sde_set_tuning(self._ctx, int(block_threads), int(grid_blocks)))

    def set_paths_per_thread(self, ppt=1):
        _check(self._ctx, lib().sde_set_paths_per_thread(self._ctx, int(ppt)))

    def set_scan_mode(self, mode=0):
        """0: automatic, 1: persistent scan kernel, 2: one point-kernel launch per point."""
        _check(self._ctx, lib().sde_set_scan_mode(self._ctx, int(mode)))

    def set_steps_per_launch(self, steps=0):
        _check(self._ctx, lib().sde_set_steps_per_launch(self._ctx, int(steps)))

    def occupancy(self, block_threads=128):
        b, s = ctypes.c_int(), ctypes.c_int()
        _check(self._ctx, lib().sde_occupancy(self._ctx, int(block_threads), ctypes.byref(b),
                                              ctypes.byref(s)))
        return b.value, s.value

    @staticmethod
    def _path_out(path_out, paths):
        po = PathOut()
        for name, want in (("X_f", 8), ("v_f", 4), ("vbar", 8), ("jP", 4), ("jD", 4)):
            t = path_out.get(name)
            if t is None:
                continue
            if not t.is_cuda or t.numel() < paths or t.element_size() != want or not t.is_contiguous():
                raise ValueError("path_out[%s] must be a contiguous CUDA tensor of %d-byte elements "
                                 "and length >= paths" % (name, want))
            setattr(po, name, t.data_ptr())
        return po

    def run(self, paths, dt, n_transient, n_avg, path_out=None, first_path=0):
        """Enqueue a run; path_out: dict of torch CUDA tensors (X_f f64, v_f f32, vbar f64,
        jP u32/i32, jD u32/i32), each of length `paths`.  first_path > 0 runs the
        realisations first_path .. first_path + paths - 1 (sde_run_range)."""
        if first_path:
            po = None if path_out is None else ctypes.byref(self._path_out(path_out, paths))
            _check(self._ctx, lib().sde_run_range(self._ctx, int(first_path), int(paths), float(dt),
                                                  int(n_transient), int(n_avg), po))
            return
        if path_out is None:
            _check(self._ctx, lib().sde_run(self._ctx, int(paths), float(dt), int(n_transient),
                                            int(n_avg)))
            return
        po = self._path_out(path_out, paths)
        _check(self._ctx, lib().sde_run_paths(self._ctx, int(paths), float(dt), int(n_transient),
                                              int(n_avg), ctypes.byref(po)))

    # segmented runs (sde_begin / sde_advance) and checkpoints

    def begin(self, paths, dt, n_transient, n_avg):
        """Start a segmented run with the current parameters and seed."""
        self._seg_paths = int(paths)
        _check(self._ctx, lib().sde_begin(self._ctx, int(paths), float(dt), int(n_transient),
                                          int(n_avg)))

    def advance(self, n_steps=0, path_out=None):
        """Enqueue one segment of n_steps steps (0: to the end); returns the steps done.
        path_out (as in run) is written by the segment that completes the run."""
        done = ctypes.c_uint64()
        po = None
        if path_out is not None:
            po = ctypes.byref(self._path_out(path_out, self._seg_paths))
        _check(self._ctx, lib().sde_advance(self._ctx, int(n_steps), po, ctypes.byref(done)))
        return done.value

    def checkpoint(self) -> bytes:
        """The segmented run's checkpoint (header and saved path states) as bytes."""
        n = ctypes.c_uint64()
        _check(self._ctx, lib().sde_checkpoint_size(self._ctx, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self._ctx, lib().sde_checkpoint(self._ctx, buf, n.value))
        return buf.raw

    def restore(self, data: bytes):
        """Continue the segmented run saved in `data` (from checkpoint())."""
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(self._ctx, lib().sde_restore(self._ctx, buf, len(data)))
        self._seg_paths = struct.unpack_from("<Q", data, 168)[0]   # header field `paths`

    def stats(self) -> dict:
        s = Stats()
        _check(self._ctx, lib().sde_stats(self._ctx, ctypes.byref(s)))
        return s.as_dict()

    def scan(self, points, deadline_ms=0.0):
        """points: list of dicts {params: Params, dt, paths, n_transient, n_avg}."""
        n = len(points)
        arr = (ScanPoint * n)()
        for i, pt in enumerate(points):
            arr[i].p = pt["params"]
            arr[i].dt = float(pt["dt"])
            arr[i].paths = int(pt["paths"])
            arr[i].n_transient = int(pt["n_transient"])
            arr[i].n_avg = int(pt["n_avg"])
        out = (Stats * n)()
        self._scan_n = n
        _check(self._ctx, lib().sde_scan(self._ctx, arr, n, out, float(deadline_ms)))
        return [o.as_dict() for o in out]

    def scan_device(self, points, out5):
        """sde_scan_device: enqueue the scan; out5 (CUDA float64 tensor of >= 5 * len(points)
        elements) receives each point's five FP64 sums.  Does not synchronise."""
        n = len(points)
        if not out5.is_cuda or out5.dtype.itemsize != 8 or out5.numel() < 5 * n or not out5.is_contiguous():
            raise ValueError("out5 must be a contiguous CUDA float64 tensor of >= 5 * npts elements")
        arr = (ScanPoint * n)()
        for i, pt in enumerate(points):
            arr[i].p = pt["params"]
            arr[i].dt = float(pt["dt"])
            arr[i].paths = int(pt["paths"])
            arr[i].n_transient = int(pt["n_transient"])
            arr[i].n_avg = int(pt["n_avg"])
        _check(self._ctx, lib().sde_scan_device(self._ctx, arr, n, ctypes.c_void_p(out5.data_ptr())))

    def scan_resume(self, deadline_ms=0.0):
        """Finish the last scan after it raised SdeTimeout (items already done are kept)."""
        n = self._scan_n
        out = (Stats * max(n, 1))()
        _check(self._ctx, lib().sde_scan_resume(self._ctx, out, float(deadline_ms)))
        return [out[i].as_dict() for i in range(n)]

    def local_error(self, paths, dt, n_steps):
        """Sec. 4's chi over paths x n_steps steps: dict of rms and max of chi_x
        (x units) and chi_v (inertial model)."""
        o = (ctypes.c_double * 4)()
        _check(self._ctx, lib().sde_local_error(self._ctx, int(paths), float(dt), int(n_steps), o))
        return {"rms_x": o[0], "rms_v": o[1], "max_x": o[2], "max_v": o[3]}

    def reduce_f64(self, vals):
        """vals: contiguous CUDA float64 tensor -> (n, sum, sum of squares)."""
        if not vals.is_cuda or vals.dtype.itemsize != 8 or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous CUDA float64 tensor")
        out = (ctypes.c_double * 3)()
        _check(self._ctx, lib().sde_reduce_f64(self._ctx, ctypes.c_void_p(vals.data_ptr()),
                                               vals.numel(), out))
        return tuple(out)

    def philox_words(self, ctr, seed):
        """ctr: (n, 4) uint32 array of counters -> (n, 4) uint32 words (device Philox)."""
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
        out = np.zeros_like(ctr)
        _check(self._ctx, lib().sde_philox_words(self._ctx, ctr.ctypes.data, ctr.shape[0],
                                                 int(seed), out.ctypes.data))
        return out


NOALLOC_MAX_PATHS = 1 << 21


def run_noalloc(model, params: Params, seed, paths, dt, n_transient, n_avg, out5, status=None,
                stream=None):
    """sde_run_noalloc: a run that allocates nothing, for callers that cannot allocate
    device memory.  out5: caller-owned CUDA float64 tensor of 5 elements (the FP64
    sums); status: optional CUDA int32 tensor of 1 element.  Enqueues and returns."""
    if not out5.is_cuda or out5.dtype.itemsize != 8 or out5.numel() < 5:
        raise ValueError("out5 must be a CUDA float64 tensor of >= 5 elements")
    st = None if status is None else ctypes.c_void_p(status.data_ptr())
    rc = lib().sde_run_noalloc(int(model), ctypes.byref(params), int(seed), int(paths), float(dt),
                               int(n_transient), int(n_avg), _stream_handle(stream),
                               ctypes.c_void_p(out5.data_ptr()), st)
    if rc != SDE_OK:
        raise SdeError(rc, lib().sde_last_error(None).decode())


def version():
    return lib().sde_version().decode()
