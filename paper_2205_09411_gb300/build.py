"""Builds the CUDA library libgmg.so in-tree for sm_103a (GB300).

The translation units are compiled in parallel by nvcc and linked into one
shared library with a plain C ABI (include/gmg.h):

* csrc/gmg_api.cu      - kernels, V-cycle schedule, solve loops, C entry points
* csrc/tree_setup.cpp  - block tree and boundary set-up on the host
  (-ffp-contract=off: the level-set arithmetic is plain IEEE)
* csrc/cluster_tail.cu - the bottom of the V-cycle on a thread-block cluster
* csrc/setup_dev.cu    - boundary detection of built-in level sets on the device
  (--fmad=false: the same arithmetic as the host set-up)
* csrc/noalloc.cu      - residual norm with a static scratch array (no allocation)
* csrc/forest.cpp      - forests of independent trees (host)
* csrc/solve_history.cpp - the solve loop with its residual history (host)
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]
SOURCES = ["gmg_api.cu", "cluster_tail.cu", "setup_dev.cu", "tree_setup.cpp", "noalloc.cu", "forest.cpp",
           "solve_history.cpp"]
# device code whose arithmetic must equal the host set-up's: no multiply-add contraction
NO_FMAD = {"setup_dev.cu"}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "gmg.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT, src + ".o")
        cmd = [nvcc] + ARCH + COMMON + (["--fmad=false"] if src in NO_FMAD else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + COMMON + ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    for p, cmd in procs:
        if p.wait() != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
