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
