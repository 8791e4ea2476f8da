"""Compiles the CUDA library in-tree: csrc/*.cu -> libgf2.so (sm_103a only).

Each translation unit is compiled in parallel with nvcc, then linked into a
shared library next to this file.  Nothing is installed anywhere else.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgf2.so")
OBJDIR = os.path.join(HERE, "_build")
# the op-counting variant (same ABI; its kernels count word operations, see
# gf2_op_counts in include/gf2.h): built only on request
COUNT_OUT = os.path.join(HERE, "libgf2_count.so")
COUNT_OBJDIR = os.path.join(HERE, "_build_count")
# the trace variant (same ABI; its decomposition kernels stamp a device
# timeline, see gf2_trace_read): built only on request
TRACE_OUT = os.path.join(HERE, "libgf2_trace.so")
TRACE_OBJDIR = os.path.join(HERE, "_build_trace")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(os.path.dirname(HERE), "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgf2.so")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(os.path.dirname(HERE), "include", "gf2.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, counting: bool = False,
          trace: bool = False) -> str:
    """Builds libgf2.so, or with counting=True the op-counting variant
    libgf2_count.so (-DGF2_COUNT_OPS), or with trace=True the trace variant
    libgf2_trace.so (-DGF2_TRACE); returns the library's path."""
    if counting and trace:
        raise ValueError("one variant at a time")
    out, objdir = (COUNT_OUT, COUNT_OBJDIR) if counting else (TRACE_OUT, TRACE_OBJDIR) if trace else (OUT, OBJDIR)
    if not force and not _stale(out):
        return out
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    extra = (extra or []) + (["-DGF2_COUNT_OPS"] if counting else []) + (["-DGF2_TRACE"] if trace else [])

    def one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(one, sources()))
    tmp = out + ".tmp"
    cmd = [cc, *ARCH, "-shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":  # pragma: no cover
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, counting="--counting" in sys.argv,
                trace="--trace" in sys.argv))
