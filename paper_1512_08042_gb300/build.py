"""Build libdsmclbm.so for sm_103a with nvcc, in-tree (paper_1512_08042_gb300/_build/).

The translation units are compiled in parallel and linked into one shared library with the
CUDA runtime linked statically. The DSMC and mapping kernels are compiled without FMA
contraction (-fmad=false; host code -ffp-contract=off) so that float positions, cell keys,
collision pairs and post-collision velocities are the IEEE results of the written expressions;
the LBM kernel keeps FMA, its results are compared with a tolerance.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libdsmclbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
UNITS = {
    "runtime.cu": ["-fmad=false"],
    "k_dsmc.cu": ["-fmad=false"],
    "k_map.cu": ["-fmad=false"],
    "k_lbm.cu": ["-fmad=true"],
    "batch.cu": ["-fmad=false"],
}
HEADERS = [os.path.join(CSRC, "hyb_internal.cuh"), os.path.join(CSRC, "dsmc_move.cuh"),
           os.path.join(INCLUDE, "dsmclbm.h")]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsmclbm.so")


def _common():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                   "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC,
                   "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + HEADERS + [__file__])


def build(force=False, verbose=False, extra=()):
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = nvcc()
    jobs = []
    objs = []
    for unit, flags in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, src):
            jobs.append([exe] + _common() + flags + list(extra) + ["-c", src, "-o", obj])
    if jobs:
        def run(cmd):
            if verbose:
                print(" ".join(cmd), flush=True)
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
            return r.stderr
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for err in ex.map(run, jobs):
                if verbose and err:
                    print(err, file=sys.stderr)
    if force or jobs or not os.path.exists(LIB):
        cmd = [exe] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-cudart", "static"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
