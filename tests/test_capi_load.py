"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/*.h declares, and rejects bad arguments before touching the GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(sde_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1409_4923_gb300 import build
    build.build()
    from paper_1409_4923_gb300 import engine
    return engine.lib()


def test_header_declares_entry_points():
    names = _declared_functions()
    for want in ("sde_create", "sde_run", "sde_stats", "sde_scan", "sde_destroy", "sde_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version(lib):
    assert b"sm_103a" in lib.sde_version()


def test_create_rejects_bad_params_without_gpu(lib):
    from paper_1409_4923_gb300 import engine as E
    ctx = ctypes.c_void_p()
    bad = [E.make_params(gamma=float("nan")),
           E.make_params(gamma=1.0, Q=-1.0),
           E.make_params(gamma=0.0),
           E.make_params(gamma=1.0, noise_flags=2),            # Poisson without lambda, zeta
           E.make_params(gamma=1.0, noise_flags=4, mua=1.0),   # dichotomous without mub
           E.make_params(gamma=1.0, noise_flags=64),
           E.make_params(gamma=1.0, point=1 << 30)]
    for p in bad:
        rc = lib.sde_create(ctypes.byref(ctx), 0, ctypes.byref(p), 0, None)
        assert rc == E.SDE_EINVAL, lib.sde_last_error(None)
    rc = lib.sde_create(ctypes.byref(ctx), 7, ctypes.byref(E.make_params(gamma=1.0)), 0, None)
    assert rc == E.SDE_EINVAL
    assert lib.sde_create(None, 0, ctypes.byref(E.make_params(gamma=1.0)), 0, None) == E.SDE_EINVAL


def test_null_context_calls(lib):
    from paper_1409_4923_gb300 import engine as E
    assert lib.sde_run(None, 10, 0.1, 0, 10) == E.SDE_EINVAL
    assert lib.sde_stats(None, None) == E.SDE_EINVAL
    lib.sde_destroy(None)


def test_surrogate_calls_reject_a_null_network(lib):
    from paper_1409_4923_gb300 import engine as E, surrogate as S
    L = S._lib()
    f = ctypes.c_float
    assert L.sde_mlp_fit(None, None, None, 16, 2, 8, f(1e-3), f(1e-4), f(0.9), f(0.999), f(1e-8), 0,
                         None) == E.SDE_EINVAL
    assert L.sde_mlp_train_step(None, None, None, 8, f(1e-3), f(0.9), f(0.999), f(1e-8), None) == E.SDE_EINVAL
    assert L.sde_mlp_forward(None, None, 8, None) == E.SDE_EINVAL
    assert L.sde_mlp_create(None, 0, None) == E.SDE_EINVAL


def test_engine_has_no_cpu_fallback(monkeypatch):
    """Without the built library the binding raises instead of computing."""
    from paper_1409_4923_gb300 import engine as E
    monkeypatch.setattr(E, "_lib", None)
    monkeypatch.setattr(E, "LIB_PATH", os.path.join(ROOT, "does-not-exist.so"))
    with pytest.raises(ImportError):
        E.lib()
