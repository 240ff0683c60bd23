"""In-tree build of the CUDA library (libspm_gb300.so) for sm_103a.

Compiles every translation unit of ``csrc/`` with nvcc in parallel and links
one shared library next to this file. Used by ``__graft_entry__.build()``.

Instrumentation builds (``--counters``: work counters, ``--clocks``: per-phase
SM clocks) go to separate libraries, libspm_gb300_counters.so and
libspm_gb300_clocks.so, that add the ``spm_debug_*`` readers; select one for a
process with the SPM_GB300_LIB environment variable. The product library
compiles the instrumentation out.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspm_gb300.so")
SOURCES = ["spm_prep.cpp", "spm_vertex.cu", "spm_flood.cu", "spm_pixel.cu", "spm_grad.cu", "spm_sources.cu", "spm_sequential.cu", "spm_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(HERE, "..", "include", "spm.h"))
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


VARIANTS = {None: ("", ()), "counters": ("_counters", ("-DSPM_COUNT",)), "clocks": ("_clocks", ("-DSPM_TIME",))}


def build(force: bool = False, verbose: bool = False, extra=(), variant=None) -> str:
    suffix, defs = VARIANTS[variant]
    lib = os.path.join(HERE, f"libspm_gb300{suffix}.so")
    bdir = os.path.join(BUILD, variant) if variant else BUILD
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(bdir, exist_ok=True)
    extra = (*defs, *extra)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stderr or r.stdout):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    # a shared library links with unresolved symbols; refuse one that has any
    # of our own (a declaration left without a definition)
    und = subprocess.run(["nm", "-uC", tmp], capture_output=True, text=True).stdout
    missing = [ln.strip() for ln in und.splitlines() if "spm" in ln]
    if missing:
        os.remove(tmp)
        raise RuntimeError("unresolved library symbols: " + "; ".join(missing))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    variant = "counters" if "--counters" in sys.argv else ("clocks" if "--clocks" in sys.argv else None)
    print(build(force="--force" in sys.argv, verbose=True,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else (), variant=variant))
