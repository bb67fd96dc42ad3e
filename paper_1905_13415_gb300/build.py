"""Builds ``libparparaw.so`` in place with nvcc for sm_103a.

The translation units are compiled in parallel (one per tile shape plus the
host / ABI unit) and linked into one shared library next to this file.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libparparaw.so")
# profiling variant: the same sources with per-phase cycle counters compiled in
PHASE_BUILD = os.path.join(HERE, "_build_phase")
PHASE_LIB = os.path.join(HERE, "libparparaw_phase.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["pp_host.cu", "pp_rows.cu", "pp_stream.cu"] + [f"pp_tile_{s}.cu" for s in ("tiny", "small", "mid", "wide", "m128", "m128x6", "s128", "mid3", "y96", "t448", "w48", "big3", "q384", "q448")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "parparaw.h"),
                                                               os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, verbose: bool, build_dir: str = BUILD, defines=()) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
           *[f"-D{d}" for d in defines], "-I", CSRC, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if verbose:
        sys.stderr.write(res.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, phase_timing: bool = False) -> str:
    lib, bdir = (PHASE_LIB, PHASE_BUILD) if phase_timing else (LIB, BUILD)
    defines = ("PP_PHASE_TIMING",) if phase_timing else ()
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, bdir, defines), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
