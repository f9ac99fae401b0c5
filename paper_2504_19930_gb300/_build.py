"""Build libpfreg.so (the CUDA kernels and the C ABI) for sm_103a with nvcc.

Sources are compiled in parallel into ``_build/`` inside the package and
linked into one shared library; nothing is installed elsewhere.

The debug library ``libpfreg_debug.so`` is the same library with the
measurement, warp and C-ABI translation units compiled with -DPF_DEBUG=1:
every gather index of the measurement and warp kernels is checked against its
buffer before the load (an index outside is counted and the load skipped;
``pf_debug_bounds`` reports it).  The other objects are shared with the
release build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libpfreg.so")
LIB_DEBUG = os.path.join(BUILD, "libpfreg_debug.so")
SOURCES = ["api.cu", "measure.cu", "filter.cu", "warp.cu", "noalloc.cu", "nn.cu", "proposal.cu", "probe.cu",
           "conv.cu", "dgrad.cu"]
DEBUG_SOURCES = ["api.cu", "measure.cu", "warp.cu"]   # the ones PF_DEBUG changes
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "pfreg.h"))
    return out


def _fresh(lib) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def up_to_date(debug: bool = False) -> bool:
    return _fresh(LIB) and (not debug or _fresh(LIB_DEBUG))


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, (r.stdout + r.stderr)


def _link(nvcc, objs, lib):
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compile and link; returns the release library's path.  Skips work when
    fresh.  debug=True also builds libpfreg_debug.so (in the same parallel
    compile).  Extra nvcc flags may also come from the PFREG_NVCC_FLAGS
    environment variable (kernel variants for A/B timing); they force a
    rebuild."""
    env_flags = os.environ.get("PFREG_NVCC_FLAGS", "").split()
    extra_flags = list(extra_flags) + env_flags
    if extra_flags:
        force = True
    if not force and up_to_date(debug):
        return LIB
    os.makedirs(os.path.join(BUILD, "dbg"), exist_ok=True)
    nvcc = _nvcc()
    jobs = [(src, os.path.join(BUILD, os.path.splitext(src)[0] + ".o"), extra_flags) for src in SOURCES]
    if debug:
        jobs += [(src, os.path.join(BUILD, "dbg", os.path.splitext(src)[0] + ".o"), extra_flags + ["-DPF_DEBUG=1"])
                 for src in DEBUG_SOURCES]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        done = list(ex.map(lambda j: _compile(nvcc, *j), jobs))
    if verbose:
        for _, log in done:
            if log:
                print(log)
    rel = [os.path.join(BUILD, os.path.splitext(src)[0] + ".o") for src in SOURCES]
    _link(nvcc, rel, LIB)
    if debug:
        dbg = [os.path.join(BUILD, "dbg", os.path.splitext(src)[0] + ".o") if src in DEBUG_SOURCES
               else os.path.join(BUILD, os.path.splitext(src)[0] + ".o") for src in SOURCES]
        _link(nvcc, dbg, LIB_DEBUG)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
