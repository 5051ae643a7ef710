"""The allocation-free totals entry point against hlbm_diag.

hlbm_population_sums_noalloc serves callers that must not allocate device
memory while they run: its scratch is a static device array inside the
library instead of the context's workspace.  Without a body force its totals
are the same quantities hlbm_diag reports, so the two must agree to the
FP32-per-node rounding the diagnostics tests allow (1e-6 relative), here on
two calls in a row.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300 import abi
    from paper_2411_10751_gb300.solver import HLBM
    return abi, HLBM


def test_noalloc_totals_match_diag_on_two_calls(mods):
    abi, HLBM = mods
    c = W.thermal_decay(nx=96, ny=80, tau_hat=0.7, Pr=0.71)   # no body force
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g.init(c.rho, c.u, c.theta)
    g.step(10)                 # even step count: the state is the first buffer of the bound arena
    state = C.c_void_p(g._arena.data_ptr())
    stream = C.c_void_p(abi.hlbm_get_stream(g.ctx))
    for call in range(2):
        ref = g.diag()         # synchronises the context's stream
        out = (C.c_double * 5)()
        st = abi.hlbm_population_sums_noalloc(abi.HLBM_D2Q37, c.nodes, abi.HLBM_F32, c.params["rho0"],
                                              state, stream, out)
        assert st == abi.HLBM_OK
        got = np.array(out[:4])
        assert abs(got[0] - ref[0]) < 1e-6 * ref[0], (call, got, ref)
        assert np.abs(got[1:3] - ref[1:3]).max() < 1e-6 * ref[0], (call, got, ref)
        assert abs(got[3] - ref[3]) < 1e-6 * ref[3], (call, got, ref)
        g.step(2)
    g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(mods):
    abi, _ = mods
    out = (C.c_double * 5)()
    too_many = 33554432 + 1
    st = abi.hlbm_population_sums_noalloc(abi.HLBM_D2Q37, too_many, abi.HLBM_F32, 1.0, C.c_void_p(16), None, out)
    assert st == abi.HLBM_EINVAL
