"""Build the engine's CUDA library (libsde.so) in-tree for sm_103a.

nvcc compiles each translation unit in parallel (-gencode
arch=compute_103a,code=sm_103a, -O3, -lineinfo) and links one shared
library; no cmake, no torch extension machinery.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsde.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = ["point_inertial.cu", "point_overdamped_washboard.cu", "point_overdamped_pwl.cu",
         "point_inertial_x2.cu", "point_overdamped_washboard_x2.cu", "point_overdamped_pwl_x2.cu",
         "segment_m0.cu", "segment_m1.cu", "segment_m2.cu", "chi_m0.cu", "chi_m1.cu", "chi_m2.cu",
         "aux_kernels.cu", "scan_x2.cu", "capi.cu", "noalloc.cu", "mlp.cu", "mlp_tc.cu"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the engine needs the CUDA toolkit to build")
    return path


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return deps


def build(force=False, verbose=False):
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_unit(u):
        obj = os.path.join(OUT_DIR, u.replace(".cu", ".o"))
        cmd = [nvcc()] + flags + ["-c", os.path.join(CSRC, u), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (u, res.stderr[-6000:]))
        return obj, res.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
