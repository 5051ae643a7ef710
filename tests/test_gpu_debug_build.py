"""The bounds-checked debug build (HLBM_DEBUG, libhlbm_debug.so) on small runs
of every kernel family (tests/debug_cases.py): no gathered, staged, frame,
store or TMA-box index leaves its buffer (the library's bounds record stays
empty), and the results equal the release library's bit for bit (the checks
touch indices only, never the arithmetic).

Both libraries run in child processes, since the binding loads one library
per process (HLBM_LIBRARY selects it at import).
"""
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = Path(__file__).resolve().parent


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import importlib
    B = importlib.import_module("paper_2411_10751_gb300.build")
    B.build()
    B.build(debug=True)
    out = {}
    for lib in ("debug", "release"):
        path = tmp_path_factory.mktemp(lib) / "res.npz"
        env = dict(os.environ, HLBM_LIBRARY=lib)
        r = subprocess.run([sys.executable, str(HERE / "debug_cases.py"), str(path)], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
        out[lib] = dict(np.load(path))
    return out


def _case_names():
    sys.path.insert(0, str(HERE))
    import debug_cases
    return list(debug_cases.cases())


@pytest.mark.parametrize("name", _case_names())
def test_debug_build_records_no_bad_index_and_matches_release(results, name):
    rel, dbg = results["release"], results["debug"]
    assert bool(dbg["debug"][0]) and not bool(rel["debug"][0])
    rec = dbg[f"{name}/record"]
    assert rec[0] == 0, f"{name}: {rec[0]} rejected accesses, first at site {rec[1]} index {rec[2]} bound {rec[3]}"
    keys = sorted(k for k in rel if k.startswith(name + "/") and not k.endswith("/record"))
    assert keys
    for k in keys:
        assert np.array_equal(rel[k], dbg[k]), (k, float(np.abs(rel[k] - dbg[k]).max()))
