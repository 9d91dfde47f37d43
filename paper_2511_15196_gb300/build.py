"""Builds libphi4smc.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each translation unit compiles in parallel; the shared library links against the
shared CUDA runtime so that it shares the process's primary context with PyTorch.

An object is reused only when a stamp beside it records the same content hash of its
source, every header of the library, the compiler flags and the nvcc binary, so
objects carried over from another machine or an older tree are rebuilt. `clean=True`
deletes every object and the library first and compiles everything from scratch.
"""
import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libphi4smc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "phi4smc.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-diag-suppress", "177"]
SOURCES = ["capi.cu", "ns.cu", "kernels_rng.cu", "kernels_lattice.cu", "kernels_temper.cu", "kernels_resample.cu",
           "kernels_cov.cu", "kernels_chol.cu", "kernels_gemm_simt.cu", "kernels_tc.cu", "kernels_ns.cu",
           "resample_static.cu", "kernels_irmh.cu", "kernels_obs.cu", "batch.cu"]


def nvcc():
    cand = os.environ.get("NVCC") or os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _digest(paths, extra):
    h = hashlib.sha256()
    for p in paths:
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update("\0".join(extra).encode())
    return h.hexdigest()


def _headers():
    return sorted(os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))) + [HEADER]


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    stamp = obj + ".stamp"
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    key = _digest([os.path.join(CSRC, src)] + _headers(), cmd + [os.path.realpath(cmd[0])])
    if os.path.exists(obj) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == key:
                return obj, False
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    with open(stamp, "w") as f:
        f.write(key + "\n")
    return obj, True


def clean():
    """Removes the library and every object and stamp of this build."""
    if os.path.isdir(BUILD):
        for name in os.listdir(BUILD):
            if name.endswith((".o", ".o.stamp")):
                os.remove(os.path.join(BUILD, name))
    if os.path.exists(LIB):
        os.remove(LIB)


def build(verbose=False, clean_first=False):
    if clean_first:
        clean()
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(_compile, SOURCES))
    objs = [o for o, _ in results]
    if not os.path.exists(LIB) or any(fresh for _, fresh in results) or \
            os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    if verbose:
        print("built", LIB, "(%d of %d objects compiled)" % (sum(f for _, f in results), len(results)))
    return LIB


if __name__ == "__main__":
    build(verbose=True, clean_first="--clean" in sys.argv)
    sys.exit(0)
