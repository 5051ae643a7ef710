"""Schedule autotuner for the fused step.

A schedule is (tile rows, nodes per thread, persistent CTAs: 1 off, 2 on,
3 multi-step) as accepted by hlbm_set_tile.  For a given domain the tuner times each candidate on the
device with CUDA events (a throwaway context on the same sizes and sources,
outside any measured region) and keeps the fastest; results are cached per
GPU, lattice, source kind, storage and size in _build/autotune.json.
"""
from __future__ import annotations

import json
from pathlib import Path

import torch

from .solver import HLBM

CACHE = Path(__file__).resolve().parent / "_build" / "autotune.json"

# the multi-step schedule (persistent = 3) is left out: on GB300 it measured
# slower than one launch per step on every workload tried (its per-tile
# release and acquire fences cost more than the launch boundary)
CANDIDATES_2D = [(8, 2, 1), (8, 1, 1), (16, 2, 1), (16, 1, 1), (4, 1, 1), (8, 2, 2), (8, 1, 2)]
CANDIDATES_3D = [(8, 2, 2), (8, 2, 1), (8, 1, 1), (4, 1, 1)]


def _key(lattice, nx, ny, nz, params, storage) -> str:
    kind = "sc" if params.get("SC") else ("thermal" if params.get("H") else "local")
    return f"{torch.cuda.get_device_name()}|{lattice}|{kind}|{storage}|{nx}x{ny}x{nz}"


def _load() -> dict:
    try:
        return json.loads(CACHE.read_text())
    except (OSError, ValueError):
        return {}


def tune(lattice: str, nx: int, ny: int, nz: int, tau_hat: float, params: dict, rho, u, theta,
         storage: str = "f32", steps: int = 256, force=None, force_kind: str | None = None,
         use_cache: bool = True) -> tuple[int, int, int]:
    """Fastest (rows, nodes_per_thread, persistent) for this domain."""
    key = _key(lattice, nx, ny, nz, params, storage)
    cache = _load()
    if use_cache and key in cache:
        return tuple(cache[key]["schedule"])
    cands = CANDIDATES_2D if lattice == "D2Q37" else CANDIDATES_3D
    timings = {}
    for sched in cands:
        g = HLBM(lattice, nx, ny, nz, tau_hat, params, storage=storage)
        if force is not None:
            g.set_force_field(force, force_kind)
        g.set_tile(*sched)
        g.init(rho, u, theta)
        g.step(64)
        g.synchronize()
        s = g.cuda_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.step(steps)
        e1.record(s)
        e1.synchronize()
        timings[sched] = e0.elapsed_time(e1) / steps
        g.close()
    best = min(timings, key=timings.get)
    cache[key] = {"schedule": list(best), "ms_per_step": {str(k): v for k, v in timings.items()}}
    CACHE.parent.mkdir(exist_ok=True)
    CACHE.write_text(json.dumps(cache, indent=1))
    return best
