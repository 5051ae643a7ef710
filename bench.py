"""Throughput of the fused high-order lattice Boltzmann step on GB300.

Workload: D2Q37 thermal decay with the Prandtl-number source H_i, 1024 x 1024
periodic, tau^ = 0.7, Pr = 0.71 (theta = 1 + 0.01 sin(2 pi x/1024),
rho = 1/theta + 1e-6 seeded noise, u_x = 0.01 sin(2 pi y/1024)); one step =
one launch of the fused pull-collide-source kernel over all 1,048,576 nodes.

Metric: MLUPS (million lattice-node updates per second), whole job over all
ranks.  The population buffers (2 x 155 MB in FP32) are larger than the
129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|f16|bf16]
                  [--impl ours|reference] [--schedule R,N,P] [--only-device]
                  [--no-variants] [--no-extras] [--no-cpu-baseline]

Besides the headline line fields, rank 0 reports the other storages
(storage_variants), their errors against the FP64 oracle on a 256^2 copy,
and two extras: the batched step over 256 uneven domains and the adjoint
run on the 128^3 D3Q39 Taylor-Green case.

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on the host cores over a 256 x 256 sample of the same workload.
Multi-GPU (torchrun): every rank advances its own independent replica of the
domain (no data-path collective; "replicas only"), timing is max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import workloads as W  # noqa: E402

WORKLOAD = "D2Q37 thermal decay + H_i (Pr=0.71), 1024x1024 periodic, tau=0.7"
# other forward workloads (--workload, and the forward_sweep extra)
WORKLOADS = {
    "thermal1024": (lambda: W.thermal_decay(n=1024), WORKLOAD),
    "kolmogorov2048": (lambda: W.kolmogorov(2048), "D2Q37 Kolmogorov flow, 2048x2048 periodic, tau=0.8, g=1e-5"),
    "kolmogorov4096": (lambda: W.kolmogorov(4096), "D2Q37 Kolmogorov flow, 4096x4096 periodic, tau=0.8, g=1e-5"),
    "tg3d128": (lambda: W.taylor_green_3d(n=128), "D3Q39 compressible Taylor-Green 128^3, Ma=0.3, tau=0.6, body force"),
    "thermal2048": (lambda: W.thermal_decay(n=2048), "D2Q37 thermal decay + H_i (Pr=0.71), 2048x2048 periodic, tau=0.7"),
    "thermal4096": (lambda: W.thermal_decay(n=4096), "D2Q37 thermal decay + H_i (Pr=0.71), 4096x4096 periodic, tau=0.7"),
    "kolmogorov1024": (lambda: W.kolmogorov(1024), "D2Q37 Kolmogorov flow, 1024x1024 periodic, tau=0.8, g=1e-5"),
    "tg3d256": (lambda: W.taylor_green_3d(n=256), "D3Q39 compressible Taylor-Green 256^3, Ma=0.3, tau=0.6, body force"),
    "droplet512": (lambda: W.droplet(n=512), "D2Q37 vdW droplet 512x512 (T/Tc 0.85, k 0.01, r0 N/4), tau=0.8"),
    "droplet1024": (lambda: W.droplet(n=1024), "D2Q37 vdW droplet 1024x1024 (T/Tc 0.85, k 0.01, r0 N/4), tau=0.8"),
    # wall-bounded step (Tamm-Mott-Smith walls, two launches per step) and the
    # Carnahan-Starling pseudopotential
    "rb1024": (lambda: W.rayleigh_benard(nx=1024, ny=1026, Ra=10000.0, roll=0.01),
               "D2Q37 Rayleigh-Benard, 1024x1026 between two walls (Ra 1e4, Pr 1.41, theta 1.4 / 1.0)"),
    "csdroplet1024": (lambda: W.droplet(n=1024, r0=256.0, Tr=0.8, k=3.02, eos="cs"),
                      "D2Q37 Carnahan-Starling droplet 1024x1024 (T/Tc 0.8, k 3.02, r0 N/4), tau=0.8"),
    # the in-place (AA) step with single-pass neighbour fields
    "thermal1024_aa": (lambda: _lagged(W.thermal_decay(n=1024)), WORKLOAD + ", in place (AA), single-pass"),
    "droplet1024_aa": (lambda: _lagged(W.droplet(n=1024)),
                       "D2Q37 vdW droplet 1024x1024 (T/Tc 0.85, k 0.01, r0 N/4), tau=0.8, in place (AA), single-pass"),
    "kolmogorov4096_aa": (lambda: _lagged(W.kolmogorov(4096)),
                          "D2Q37 Kolmogorov flow, 4096x4096 periodic, tau=0.8, g=1e-5, in place (AA)"),
}


def _lagged(case):
    case.params = dict(case.params)
    case.params["lag"] = True
    return case


def _bytes_per_node(case, storage):
    """Algorithmic bytes per lattice update: one read and one write of every
    population (+ the in-place step's neighbour field, written and read once)."""
    b = 2 * (37 if case.lattice == "D2Q37" else 39) * (4 if storage == "f32" else 2)
    if case.params.get("lag") and (case.params.get("H") or case.params.get("SC")):
        b += 8
    return b


def _set_force(g, case):
    if case.gfield is not None:
        if case.lattice == "D2Q37":
            g.set_force_field(case.gfield[:, :, 0], "profile")
        else:
            g.set_force_field(case.gfield, "field")
METRIC = "MLUPS"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, lrank


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that define the 2D fused step kernels (what the DRAM counters describe)
STEP2D_SOURCES = ("step2d.cuh", "step_common.cuh", "tma.cuh", "lattice.cuh", "lattice_gen.cpp", "internal.h",
                  "step2d_f32.cu", "step2d_f16.cu", "step2d_bf16.cu", "aa.cu")


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in STEP2D_SOURCES:
        h.update((ROOT / "paper_2411_10751_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def _multistep(case, sched) -> bool:
    """Whether this schedule runs the multi-step kernel on this workload
    (D2Q37, persistent = 3, tiles covering the domain exactly)."""
    if case.lattice != "D2Q37" or sched[2] != 3:
        return False
    h = 3 if case.params.get("SC") else (1 if case.params.get("H") else 0)
    return case.nx % 32 == 0 and case.ny % sched[0] == 0 and h + 3 <= sched[0]


def _launches(case, sched, steps) -> int:
    """Step-kernel launches of hlbm_step(steps): one per step, or one per
    block of up to 1024 steps for the multi-step kernel."""
    if case.params.get("walls"):
        return 3 * steps   # wall completion, moments, collision
    if not _multistep(case, sched):
        return steps
    tiles = (case.nx // 32) * (case.ny // sched[0])
    smax = max(1, min(1024, (2 ** 31 - 1) // tiles))
    return -(-steps // smax)


def _ncu_traffic(kernel_hash: str, storage: str, schedule, workload: str = "thermal1024"):
    """DRAM bytes per step of the fused kernel from the committed ncu summary
    (a range capture over consecutive steps), if it was captured from the
    current kernel sources on this workload with this schedule; else None."""
    p = ROOT / "profiles" / "fused_step_thermal1024_dram.json"
    if not p.exists():
        return None
    try:
        d = json.loads(p.read_text())
    except ValueError:
        return None
    if d.get("kernel_source_sha") != kernel_hash:
        return None
    for e in d.get("entries", []):
        if (e.get("storage") == storage and list(e.get("schedule", [])) == list(schedule)
                and e.get("workload", "thermal1024") == workload):
            # multi-step entries: one launch runs several steps; the figure is per step
            return e.get("dram_bytes_per_step", e.get("dram_bytes_per_launch"))
    return None


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region.

    A thread reads NVML (libnvidia-ml through ctypes) every few milliseconds
    while the region runs, plus one sample right before and one right after,
    so even a region of a few milliseconds has samples; where NVML cannot be
    loaded, nvidia-smi is polled every 100 ms instead."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int, period_s: float = 0.002):
        self.gpu = gpu_index
        self.period = period_s
        self.rows = []            # (sm_mhz, max_mhz, reason bits)
        self.proc = None
        self.path = None
        self._nvml = None
        self._h = None
        self._thread = None
        self._stop = None

    def _nvml_open(self):
        import ctypes as C
        try:
            lib = C.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if lib.nvmlInit_v2() != 0:
            return False
        h = C.c_void_p()
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        ok = -1
        if ids and self.gpu < len(ids):
            tok = ids[self.gpu]
            if tok.isdigit():
                ok = lib.nvmlDeviceGetHandleByIndex_v2(int(tok), C.byref(h))
            else:
                ok = lib.nvmlDeviceGetHandleByUUID(tok.encode(), C.byref(h))
        else:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(self.gpu, C.byref(h))
        if ok != 0:
            return False
        self._nvml, self._h = lib, h
        return True

    def sample(self):
        import ctypes as C
        if self._nvml is None:
            return
        mhz, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        lib = self._nvml
        if lib.nvmlDeviceGetClockInfo(self._h, 1, C.byref(mhz)) != 0:      # NVML_CLOCK_SM
            return
        lib.nvmlDeviceGetMaxClockInfo(self._h, 1, C.byref(mx))
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self._h, C.byref(rs))
        self.rows.append((float(mhz.value), float(mx.value), int(rs.value)))

    def _loop(self):
        while not self._stop.is_set():
            self.sample()
            self._stop.wait(self.period)

    def __enter__(self):
        import threading
        if self._nvml_open():
            self._stop = threading.Event()
            self.sample()
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
            return self
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()
            self.sample()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            bits = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                    "sw_power_cap": 0x4}
            if self.path and os.path.exists(self.path):
                for line in open(self.path):
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        r = sum(bits[names[k]] for k in range(4) if parts[5 + k].lower() == "active")
                        self.rows.append((float(parts[1]), float(parts[2]), r))
                    except ValueError:
                        continue
                os.unlink(self.path)

    def summary(self):
        if not self.rows:
            return None
        reasons = sorted({name for _, _, r in self.rows for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": max(r[1] for r in self.rows),
                "sm_mhz_min": min(r[0] for r in self.rows), "reasons": reasons, "samples": len(self.rows),
                "source": "nvml" if self._nvml is not None else "nvidia-smi"}


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_items: int, rank: int, ws: int) -> list[int]:
    """Round-robin share of n independent items for this rank."""
    return list(range(rank, n_items, ws))


def tuned_schedule(case, storage, lrank):
    """Autotuned (rows, nodes per thread, persistent) for this workload (untimed)."""
    import torch
    from paper_2411_10751_gb300 import autotune
    force, kind = None, None
    if case.gfield is not None:
        force, kind = (case.gfield[:, :, 0], "profile") if case.lattice == "D2Q37" else (case.gfield, "field")
    with torch.cuda.device(lrank):
        return autotune.tune(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params,
                             case.rho, case.u, case.theta, storage=storage, force=force, force_kind=kind)


def forward_sweep(lrank, steps=400, warmup=20):
    """The other forward configurations measured against the HBM roofline: the
    Kolmogorov flow at 2048^2 and 4096^2 and the D3Q39 Taylor-Green 128^3 step."""
    peak, kind = _peaks()
    out = []
    for name in ("kolmogorov2048", "kolmogorov4096", "tg3d128"):
        case = WORKLOADS[name][0]()
        sched = tuned_schedule(case, "f32", lrank)
        ms, _, _, _ = time_device(case, "f32", steps, warmup, 1, lrank, sched)
        mlups = case.nodes * steps / (ms * 1e-3) / 1e6
        gbs = _bytes_per_node(case, "f32") * mlups / 1e3
        out.append({"workload": WORKLOADS[name][1], "storage": "f32", "schedule": list(sched), "MLUPS": mlups,
                    "achieved_GBs": gbs, "frac_of_" + kind: gbs / peak})
    return out


REPEATS = 5


def time_device(case, storage, steps, warmup, ws, lrank, schedule=None, repeats=REPEATS):
    """Device-resident run: W warm-up steps, then `repeats` timed regions of
    exactly K steps, each bracketed by a barrier and a device synchronize and
    timed with CUDA events on the context's stream; returns the median region
    (ms), the clock record over all regions, the FP64 diagnostics and every
    region's time."""
    import torch
    from paper_2411_10751_gb300.solver import HLBM
    g = HLBM(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params, storage=storage, device=lrank)
    if schedule:
        g.set_tile(*schedule)
    _set_force(g, case)
    g.init(case.rho, case.u, case.theta)
    g.step(warmup)
    g.synchronize()
    s = g.cuda_stream()
    times = []
    with ClockSampler(lrank) as clk:
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            _barrier(ws)
            torch.cuda.synchronize()
            e0.record(s)
            g.step(steps)
            e1.record(s)
            e1.synchronize()
            torch.cuda.synchronize()
            _barrier(ws)
            times.append(e0.elapsed_time(e1))
    d = g.diag()
    g.close()
    return statistics.median(times), clk.summary(), d, times


def profile_window(case, storage, steps, warmup, lrank, schedule):
    """K consecutive steps after W warm-up steps, bracketed by cudaProfilerStart /
    cudaProfilerStop: under an ncu range capture without cache control the
    window starts in the steady state of the step sequence, so the dirty
    lines the window inherits balance those it leaves, and its DRAM bytes / K
    are the traffic of one step."""
    import torch
    from paper_2411_10751_gb300.solver import HLBM
    g = HLBM(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params, storage=storage, device=lrank)
    g.set_tile(*schedule)
    _set_force(g, case)
    g.init(case.rho, case.u, case.theta)
    g.step(warmup)
    g.synchronize()
    torch.cuda.profiler.start()
    g.step(steps)
    g.synchronize()
    torch.cuda.profiler.stop()
    g.close()


def time_e2e(case, storage, steps, ws, lrank, schedule=None, repeats=REPEATS):
    """Through the public API with host buffers: pinned host fields -> hlbm_init
    (H2D), K steps, hlbm_moments to pinned host buffers (D2H); wall time, the
    median of `repeats` runs."""
    import torch
    from paper_2411_10751_gb300.solver import HLBM
    g = HLBM(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params, storage=storage, device=lrank)
    if schedule:
        g.set_tile(*schedule)
    _set_force(g, case)
    pin = {k: torch.from_numpy(np.asarray(getattr(case, k), np.float32)).pin_memory() for k in ("rho", "u", "theta")}
    out = {k: torch.empty_like(pin[k]).pin_memory() for k in pin}
    g.init(pin["rho"].numpy(), pin["u"].numpy(), pin["theta"].numpy())   # warm-up of the path
    g.synchronize()
    from paper_2411_10751_gb300 import abi
    times = []
    for _ in range(repeats):
        _barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        abi.check(abi.hlbm_init(g.ctx, pin["rho"].data_ptr(), pin["u"].data_ptr(), pin["theta"].data_ptr(), 0),
                  g.ctx)
        abi.check(abi.hlbm_step(g.ctx, steps), g.ctx)
        abi.check(abi.hlbm_moments(g.ctx, out["rho"].data_ptr(), out["u"].data_ptr(), out["theta"].data_ptr(), 0),
                  g.ctx)
        t1 = time.perf_counter()
        _barrier(ws)
        times.append((t1 - t0) * 1e3)
    h2d = sum(t.numel() * 4 for t in pin.values())
    d2h = sum(t.numel() * 4 for t in out.values())
    assert np.isfinite(out["u"].numpy()).all()
    g.close()
    return statistics.median(times), h2d, d2h


def storage_errors(case, schedules, steps=100):
    """Per-field error of each storage against the FP64 oracle on the benchmark
    workload itself, each storage on the schedule its timing used."""
    from oracle.solver import Oracle
    from paper_2411_10751_gb300.solver import HLBM
    c = case
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    if c.gfield is not None:
        o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    o.run(steps)
    r0, u0, t0 = o.moments()
    res = {}
    for st, sched in schedules.items():
        g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=st)
        g.set_tile(*sched)
        _set_force(g, c)
        g.init(c.rho, c.u, c.theta)
        g.step(steps)
        r, u, t = g.moments_host()
        g.close()
        res[st] = {"rho": float(np.abs(r - r0).max() / np.abs(r0).max()),
                   "u": float(np.sqrt(((u - u0) ** 2).sum(0)).max() / np.sqrt((u0 ** 2).sum(0)).max()),
                   "theta": float(np.abs(t - t0).max() / np.abs(t0).max()), "schedule": list(sched)}
    return {"case": f"the benchmark workload ({c.nx}x{c.ny}), {steps} steps, each storage on its timed schedule, "
                    "max|q-q_oracle|/max|q_oracle|", **res}


def _oracle_mlups(o, nodes, budget_s, min_steps=1):
    o.run(1)
    t0 = time.perf_counter()
    k = 0
    while k < min_steps or time.perf_counter() - t0 < budget_s:
        o.run(1)
        k += 1
    dt = time.perf_counter() - t0
    return nodes * k / dt / 1e6, k, dt


def cpu_baseline(budget_s=10.0, n=1024):
    """FP64 oracle on the host cores over the full 1024^2 workload: as many
    whole steps as fit in about budget_s seconds on all cores (at least 2),
    and the same with one thread (at least 1 step)."""
    from oracle import solver as osol
    c = W.thermal_decay(n=n)
    o = osol.Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    o.init(c.rho, c.u, c.theta)
    cores = osol.get_threads()
    v, k, dt = _oracle_mlups(o, c.nodes, budget_s, 2)
    osol.set_threads(1)
    v1, k1, dt1 = _oracle_mlups(o, c.nodes, budget_s / 2, 1)
    osol.set_threads(cores)
    return {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{k} FP64 oracle steps of the full {n}x{n} workload ({dt:.1f} s) on {cores} threads",
            "single_thread": {"value": v1, "unit": METRIC, "cores": 1,
                              "sample": f"{k1} steps of the same workload ({dt1:.1f} s) on one thread"}}


def batched_extra(lrank, ws=1, rank=0, steps=100):
    """Batched step: 256 independent Kolmogorov/droplet domains of sides
    32..256 (hlbm_batch_*), device-resident, CUDA events on the batch stream.
    With several ranks each steps its round-robin share of the domains (no
    data exchange); the time is the maximum over ranks."""
    import torch
    from paper_2411_10751_gb300.solver import HLBM, Batch
    all_cases = W.batched(256, seed=0)
    cases = [all_cases[k] for k in shard(len(all_cases), rank, ws)]
    ctxs = []
    for c in cases:
        g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params, device=lrank)
        if c.gfield is not None:
            g.set_force_field(c.gfield[:, :, 0], "profile")
        g.init(c.rho, c.u, c.theta)
        ctxs.append(g)
    b = Batch(ctxs)
    b.step(4)
    b.synchronize()
    s = b.cuda_stream(lrank)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    e0.record(s)
    b.step(steps)
    e1.record(s)
    e1.synchronize()
    _barrier(ws)
    ms = _max_over_ranks(ws, e0.elapsed_time(e1))
    nodes = sum(c.nodes for c in all_cases)
    b.close()
    for g in ctxs:
        g.close()
    return {"workload": "256 periodic D2Q37 domains (Kolmogorov + H_i, vdW droplets), sides 32..256, FP32",
            "nodes": nodes, "steps": steps, "launches_per_rank": steps, "ranks": ws,
            "kernel": "batch_step_kernel (one persistent launch per step over every domain and kind)",
            "MLUPS": nodes * steps / (ms * 1e-3) / 1e6, "achieved_GBs": 296 * nodes / (ms * 1e-3 / steps) / 1e9}


def _adjoint_once(c, sched, lrank, steps, ckpt):
    import torch
    from paper_2411_10751_gb300.solver import HLBM
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, device=lrank)
    g.set_tile(*sched)
    g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    g.adjoint(steps, ckpt)               # warm-up: every kernel, the workspace block, the tensor maps
    g.init(c.rho, c.u, c.theta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, grad = g.adjoint(steps, ckpt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    g.close()
    del grad
    torch.cuda.empty_cache()
    return {"checkpoint_every": ckpt, "seconds": dt, "ms_per_reverse_step": dt * 1e3 / steps,
            "MLUPS_reverse": c.nodes * steps / dt / 1e6, "loss": loss}


def adjoint_extra(lrank, n=128, steps=400, ckpt=None):
    """Adjoint of the body-force step on the D3Q39 Taylor-Green case
    (hlbm_adjoint_run), checkpoint every 50 steps (the configuration's
    interval; ckpt overrides it).  When every state fits in HBM, the same run
    with interval 1 (no checkpoint copies, no recompute) is reported beside it."""
    import torch
    from paper_2411_10751_gb300 import abi
    from paper_2411_10751_gb300.solver import HLBM
    c = W.taylor_green_3d(n=n, tau_hat=0.6, Ma=0.3, steps=steps)
    sched = tuned_schedule(c, "f32", lrank)      # forward and recompute steps
    main = _adjoint_once(c, sched, lrank, steps, ckpt or 50)
    out = {"workload": f"D3Q39 Taylor-Green {n}^3, Ma 0.3, tau 0.6: dL/dg of the kinetic energy at step {steps}, "
                       f"checkpoint every {main['checkpoint_every']}",
           "forward_schedule": list(sched), **main,
           "note": "wall time of hlbm_adjoint_run: forward steps with checkpoints, one recomputed segment at a "
                   "time, reverse steps"}
    if ckpt is None:
        g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, device=lrank)
        need = abi.hlbm_adjoint_workspace_bytes(g.ctx, steps, 1)
        g.close()
        free, _ = torch.cuda.mem_get_info(lrank)
        if need + (8 << 30) < free:
            out["every_state_kept"] = _adjoint_once(c, sched, lrank, steps, 1)
    return out


def reference_side(steps: int, rate_mlups: float = 8.0, budget_s: float = 120.0) -> int:
    """Side of the square sample of the workload the reference arm steps: the
    full 1024 when (steps + warm-up) oracle steps fit in about budget_s at the
    oracle's rate, else the largest power of two that does (at least 64)."""
    n = 1024
    while n > 64 and steps * n * n / (rate_mlups * 1e6) > budget_s:
        n //= 2
    return n


def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores,
    over the benchmark workload (or a bounded square sample of it)."""
    if rank != 0:
        return 0
    from oracle import solver as osol
    osol.build()
    n = reference_side(args.steps + args.warmup)
    c = W.thermal_decay(n=n)
    o = osol.Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    o.init(c.rho, c.u, c.theta)
    o.run(args.warmup)
    t0 = time.perf_counter()
    o.run(args.steps)
    dt = time.perf_counter() - t0
    v = c.nodes * args.steps / dt / 1e6
    sample = (f"{args.steps} FP64 oracle steps of the full {n}x{n} workload" if n == 1024 else
              f"{args.steps} FP64 oracle steps on a {n}x{n} sample of the workload (the full 1024x1024 would "
              f"exceed the time bound at this step count)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{n}x{n}",
                                            "same_config": n == 1024},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": osol.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and adjoint lines")
    ap.add_argument("--schedule", default=None, help="rows,nodes_per_thread,persistent (skips the autotuner)")
    ap.add_argument("--workload", default="thermal1024", choices=sorted(WORKLOADS),
                    help="forward workload of the line (default: the 1024^2 thermal-decay benchmark)")
    ap.add_argument("--only-device", action="store_true",
                    help="device-timed steps only (no e2e, variants, extras or CPU baseline; for profiling)")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="run the adjoint extra alone and print its line (for profiling)")
    ap.add_argument("--only-batched", action="store_true",
                    help="run the batched extra alone and print its line (for profiling)")
    ap.add_argument("--profile-range", action="store_true",
                    help="after the warm-up, run K steps between cudaProfilerStart and cudaProfilerStop and exit "
                         "(the window an ncu range capture measures)")
    ap.add_argument("--adjoint-steps", type=int, default=400, help="T of the adjoint line")
    ap.add_argument("--adjoint-ckpt", type=int, default=None,
                    help="checkpoint interval of the adjoint line (default: 1 when every state fits in HBM, else 50)")
    args = ap.parse_args()
    if args.only_device:
        args.no_variants = args.no_extras = args.no_cpu_baseline = True
    args.warmup = max(args.warmup, 3)
    ws, rank, lrank = _dist()

    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl")
    import paper_2411_10751_gb300 as pkg
    if rank == 0 or ws == 1:
        pkg.build()
    _barrier(ws)
    pkg.load()
    if args.only_batched:
        if rank == 0 or ws > 1:
            line = batched_extra(lrank, ws, rank)
            if rank == 0:
                print(json.dumps({"batched": line}))
        return 0
    if args.only_adjoint:
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_extra(lrank, steps=args.adjoint_steps, ckpt=args.adjoint_ckpt)}))
        return 0

    case = WORKLOADS[args.workload][0]()
    if args.profile_range:
        if rank == 0:
            sched = tuple(int(v) for v in args.schedule.split(",")) if args.schedule else \
                tuned_schedule(case, args.storage, lrank)
            profile_window(case, args.storage, args.steps, args.warmup, lrank, sched)
        return 0
    if args.schedule:
        sched = tuple(int(v) for v in args.schedule.split(","))
    else:
        sched = tuned_schedule(case, args.storage, lrank)
    ms, clocks, diag, region_ms = time_device(case, args.storage, args.steps, args.warmup, ws, lrank, sched)
    ms = _max_over_ranks(ws, ms)
    nodes = case.nodes
    value = nodes * args.steps * ws / (ms * 1e-3) / 1e6
    elem = 4 if args.storage == "f32" else 2
    bytes_per_node = _bytes_per_node(case, args.storage)
    launch_s = ms * 1e-3 / args.steps
    achieved = bytes_per_node * nodes / launch_s / 1e9
    peak, peak_kind = _peaks()
    khash = _kernel_source_hash()

    e2e = None
    if not args.only_device:
        e2e_ms, h2d, d2h = time_e2e(case, args.storage, args.steps, ws, lrank, sched)
        e2e_ms = _max_over_ranks(ws, e2e_ms)
        e2e = {"value": nodes * args.steps * ws / (e2e_ms * 1e-3) / 1e6, "unit": METRIC,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "path": "hlbm_init(host) + hlbm_step(K) + hlbm_moments(host), pinned host buffers"}

    variants = None
    errors = None
    cpu = None
    extras = None
    if not args.no_extras:
        extras = {"batched": batched_extra(lrank, ws, rank)}
        if rank == 0:
            extras["adjoint"] = adjoint_extra(lrank)
            extras["forward_sweep"] = forward_sweep(lrank)
    if rank == 0:
        if not args.no_variants:
            variants = {}
            vscheds = {args.storage: sched}
            for st in ("f32", "f16", "bf16"):
                if st == args.storage:
                    continue
                k = min(args.steps, 4000)
                vsched = tuned_schedule(case, st, lrank)
                vms, _, _, _ = time_device(case, st, k, args.warmup, 1, lrank, vsched)
                vscheds[st] = vsched
                e = 4 if st == "f32" else 2
                variants[st] = {"MLUPS": nodes * k / (vms * 1e-3) / 1e6, "schedule": list(vsched),
                                "achieved_GBs": _bytes_per_node(case, st) * nodes / (vms * 1e-3 / k) / 1e9,
                                "frac_of_" + peak_kind: _bytes_per_node(case, st) * nodes / (vms * 1e-3 / k) / 1e9 / peak}
            if args.workload == "thermal1024":
                errors = storage_errors(case, vscheds)
        if not args.no_cpu_baseline:
            cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1], "nodes_per_gpu": nodes, "storage": args.storage,
                       "schedule": {"rows": sched[0], "nodes_per_thread": sched[1],
                                    "persistent": sched[2] >= 2, "multi_step": _multistep(case, sched),
                                    "chosen_by": "--schedule" if args.schedule else "autotune"},
                       "parallelism": f"replicas{ws}" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (2 x %d MB population buffers), no flush" %
                             (bytes_per_node // 2 * nodes // 2 ** 20)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": _ncu_traffic(khash, args.storage, sched, args.workload),
                         "algorithmic_bytes_per_node": bytes_per_node,
                         "kernel": "wall_complete_kernel + wall_moments_kernel + wall_collide_kernel (three launches per step, the "
                                   "populations read in both)" if case.params.get("walls") else
                                   "aa_step_kernel (in place, one launch per step)" if case.params.get("lag") else
                                   (("step3d_rows_kernel" if sched[2] >= 2 and case.nx in (32, 64, 128, 256)
                                     else "step3d_kernel") if case.lattice == "D3Q39" else
                                    ("step2d_multistep_kernel" if _multistep(case, sched) else
                                     "step2d_persistent_kernel" if sched[2] >= 2 else "step2d_kernel")) +
                                   f" ({sched[0]} rows, {sched[1]} nodes per thread)" +
                                   (", one launch per up to 1024 steps: achieved and traffic per step"
                                    if _multistep(case, sched) else "")},
            "e2e": e2e,
            "gpu_launches": _launches(case, sched, args.steps),
            "timing": {"repeats": len(region_ms), "statistic": "median of the timed regions of K steps",
                       "region_ms": region_ms},
            "clocks": clocks,
            "cpu_baseline": cpu,
            "storage_variants": variants,
            "storage_error_vs_oracle": errors,
            "extras": extras,
            "final_diag": [float(x) for x in diag],
            "kernel_source_sha": khash,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
