"""Build libgsp.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then the
objects are linked into paper_2603_08661_gb300/libgsp.so.  The same sources
compiled with -DGSP_DEBUG give libgsp_debug.so, the bounds-checked build
(every guarded index is compared with its bound; an index out of bounds
records GSP_ERR_CAPACITY instead of touching memory).  Run it as a script
(`python paper_2603_08661_gb300/build.py`): importing the package loads the
library this builds (GSP_LIBRARY in the environment names another build).
__graft_entry__.build() loads it by path.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgsp.so")
DEBUG_OUT_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libgsp_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
              "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _variants(debug: bool):
    """(object dir, library, extra flags) of the release and the bounds-checked build."""
    out = [(OUT_DIR, LIB, [])]
    if debug:
        out.append((DEBUG_OUT_DIR, DEBUG_LIB, ["-DGSP_DEBUG"]))
    return out


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile (in parallel) and link libgsp.so, and libgsp_debug.so when debug is
    set; returns the path of libgsp.so."""
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "gsp.h"))
    nvcc = _nvcc()
    procs, links = [], []
    for out_dir, lib, extra in _variants(debug):
        os.makedirs(out_dir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
                if ptxas_info:
                    cmd.insert(1, "-Xptxas=-v")
                if verbose:
                    print(" ".join(cmd), flush=True)
                procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out and (verbose or ptxas_info or p.returncode):
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    for lib, objs in links:
        if force or _stale(lib, objs):
            tmp = lib + f".{os.getpid()}.tmp"
            subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv, debug="--debug" in sys.argv)
