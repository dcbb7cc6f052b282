"""In-tree build of libblockbp.so for sm_103a (nvcc, no CMake).

Each CUDA translation unit is compiled in parallel into ``_build/`` next to
this file, then linked into ``libblockbp.so`` inside the package directory.
Rebuilds only what is older than its sources.
"""

from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libblockbp.so")
# The same sources with device bounds checks (-DBLOCKBP_CHECKS): every table
# index the kernels derive is tested before use, failures flagged
# (BBP_FLAG_CHECK) and skipped.  Built on request only.
BUILD_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(HERE, "libblockbp_checks.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["bbp_api.cu", "bbp_decode_f64.cu", "bbp_decode_f32.cu", "bbp_fused_f32.cu", "bbp_fused_f64.cu",
           "bbp_sample.cu", "bbp_static.cu", "bbp_warm.cu", "bbp_warm_tc.cu",
           "bbp_warm_decode.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "blockbp.h"))
    return max(os.path.getmtime(f) for f in files)


def build(verbose: bool = False, force: bool = False, checks: bool = False) -> str:
    """Compile and link the library (with ``checks``, the variant with device
    bounds checks); returns its path."""
    bdir, lib_path = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    extra = ["-DBLOCKBP_CHECKS"] if checks else []
    os.makedirs(bdir, exist_ok=True)
    newest = _deps_mtime()
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= newest:
            continue
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", lib_path, *objs, "-lcudart"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, checks="--checks" in sys.argv))
