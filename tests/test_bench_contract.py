"""bench.py's output contract, on the CPU.

The reference arm (the FP64 oracle on the host cores) runs without a GPU: its
single JSON line must carry the keys and types the measurement contract
requires.  The GPU arm's helpers that decide `gpu_launches` and the multi-step
schedule are checked against their definitions.
"""
import json
import subprocess
import sys
from pathlib import Path

import bench
import workloads as W

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key, typ in [("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)]:
        assert isinstance(d[key], typ), key
    assert d["warmup"] >= 3
    assert d["vs_baseline"] is None
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_launch_count_and_multistep_rule():
    c = W.thermal_decay(n=1024)
    assert not bench._multistep(c, (8, 2, 2))
    assert bench._launches(c, (8, 2, 2), 10000) == 10000
    assert bench._multistep(c, (8, 2, 3))
    assert bench._launches(c, (8, 2, 3), 10000) == 10          # up to 1024 steps per launch
    assert bench._multistep(c, (4, 1, 3))                      # frame 1 + pull 3 fits a 4-row tile
    ragged = W.thermal_decay(nx=100, ny=75)
    assert not bench._multistep(ragged, (8, 2, 3))            # tiles do not cover the domain
    drop = W.droplet(n=512)
    assert not bench._multistep(drop, (4, 1, 3))              # frame 3 + pull 3 exceeds a 4-row tile
    assert bench._multistep(drop, (8, 1, 3))


def test_every_workload_builds_with_its_byte_count():
    """Each bench workload constructs with finite fields of its stated size;
    the algorithmic bytes per node follow the storage, the lattice and the
    in-place step's neighbour field; the wall step counts its three launches."""
    import numpy as np
    for name, (make, desc) in bench.WORKLOADS.items():
        if name in ("kolmogorov4096", "thermal4096", "tg3d256", "kolmogorov4096_aa"):
            continue   # the same constructors at a size too large for a quick CPU check
        c = make()
        assert desc and c.rho.shape == ((c.ny, c.nx) if c.lattice == "D2Q37" else (c.nz, c.ny, c.nx)), name
        for f in (c.rho, c.u, c.theta):
            assert np.isfinite(f).all(), name
        q = 37 if c.lattice == "D2Q37" else 39
        lag = 8 if c.params.get("lag") and (c.params.get("H") or c.params.get("SC")) else 0
        assert bench._bytes_per_node(c, "f32") == 2 * q * 4 + lag, name
        assert bench._bytes_per_node(c, "f16") == 2 * q * 2 + lag, name
    rb = bench.WORKLOADS["rb1024"][0]()
    assert rb.params.get("walls") and bench._launches(rb, (8, 1, 1), 20) == 60
