"""Builds libhlbm.so (the CUDA library behind include/hlbm.h) in-tree for sm_103a.

Steps: compile and run the host generator of the D2Q37 quadrature weights
(csrc/lattice_gen.cpp -> _build/lattice_weights.inc), compile every CUDA
translation unit in parallel with nvcc, link a shared library.  Output:
paper_2411_10751_gb300/_build/libhlbm.so; with debug=True (`--debug`) the
bounds-checking variant _build/debug/libhlbm_debug.so, which the binding
loads instead when HLBM_LIBRARY=debug is set.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libhlbm.so"
DEBUG_LIB = BUILD / "debug" / "libhlbm_debug.so"

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-std=c++17", "--expt-relaxed-constexpr", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
          f"-I{CSRC}", f"-I{BUILD}", f"-I{ROOT / 'include'}"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: " + " ".join(map(str, cmd)) + "\n" + r.stdout + r.stderr)
    return r


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> Path:
    """debug: the bounds-checking variant (HLBM_DEBUG) as
    _build/debug/libhlbm_debug.so."""
    BUILD.mkdir(exist_ok=True)
    gen = BUILD / "lattice_gen"
    inc = BUILD / "lattice_weights.inc"
    if force or _stale(gen, [CSRC / "lattice_gen.cpp"]):
        _run(["g++", "-O2", "-o", str(gen), str(CSRC / "lattice_gen.cpp")])
    if force or _stale(inc, [gen]):
        _run([str(gen), str(inc)])
    headers = list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + [ROOT / "include" / "hlbm.h", inc]
    out_dir, lib, extra = BUILD, LIB, []
    if debug:
        out_dir, lib, extra = DEBUG_LIB.parent, DEBUG_LIB, ["-DHLBM_DEBUG"]
        out_dir.mkdir(exist_ok=True)
    objs, jobs = [], []
    for cu in sources():
        obj = out_dir / (cu.stem + ".o")
        objs.append(obj)
        if force or _stale(obj, [cu] + headers):
            jobs.append([NVCC, *ARCH, *CFLAGS, *extra, "-c", str(cu), "-o", str(obj)])
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for r in ex.map(_run, jobs):
                if verbose and r.stderr:
                    print(r.stderr, file=sys.stderr)
    if force or jobs or _stale(lib, objs):
        _run([NVCC, *ARCH, "-shared", "-o", str(lib), *map(str, objs)])
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
