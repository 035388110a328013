"""Build libttc.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under csrc/ is compiled in parallel to an object file,
then linked into ``paper_1607_01249_gb300/libttc.so`` (static CUDA runtime, so
the library needs nothing but the driver at run time).  No cmake, no torch.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libttc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _digest(paths, extra=""):
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile (if anything changed) and return the path of libttc.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    flags = NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_verbose else [])
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest(srcs + _headers(), " ".join(ARCH + flags) + os.uname().machine)
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    cc = nvcc()
    hdr_dig = _digest(_headers(), " ".join(ARCH + flags) + os.uname().machine)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        sd = _digest([src], hdr_dig)
        st = obj + ".stamp"
        if not force and os.path.exists(obj) and os.path.exists(st) and open(st).read() == sd:
            return obj, ""
        cmd = [cc] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        with open(st, "w") as f:
            f.write(sd)
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_verbose:
        for _, log in results:
            if log:
                print(log)
    objs = [o for o, _ in results]
    tmp = LIB + f".tmp{os.getpid()}"
    # cuBLAS (the GEMM of the TTGT contractions) from the toolkit's own
    # library directory, found again at load time through the rpath
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    cmd = ([cc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs +
           ["-L", cuda_lib, "-lcublas", "-Xlinker", "-rpath", "-Xlinker", cuda_lib, "-lpthread"])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv))
