"""Build the in-tree shared libraries for sm_103a with nvcc.

``libinla_gpu.so`` is the evaluation library (include/inla_gpu.h);
``libinla_probe.so`` holds the benchmark's throughput probes
(include/inla_probe.h).  Each translation unit under ``csrc/`` is compiled in
parallel into ``_build/`` and linked in-tree (both git-ignored).  Objects are
rebuilt when a source or a header is newer.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libinla_gpu.so")
PROBE_LIB = os.path.join(PKG, "libinla_probe.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
SOURCES = ["dense_blocks.cu", "bta_kernels.cu", "setup_kernels.cu", "capi.cu", "tc_gemm.cu", "ozaki.cu", "synth.cpp"]
PROBE_SOURCES = ["probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-I", INCLUDE]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; returns the library path.  Raises on compiler errors."""
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()
    hdr = _headers_mtime()
    jobs = []
    for src in SOURCES + PROBE_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}:\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(max_workers=len(SOURCES) + len(PROBE_SOURCES)) as ex:
        list(ex.map(run, jobs))
    for lib, srcs in ((LIB, SOURCES), (PROBE_LIB, PROBE_SOURCES)):
        objs = [os.path.join(OBJDIR, os.path.splitext(s)[0] + ".o") for s in srcs]
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
            tmp = lib + ".tmp"
            run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
