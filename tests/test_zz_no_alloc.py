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


def _case(lattice):
    """A state with net momentum in every direction (a uniform drift on top of
    the workload's field), no body force."""
    if lattice == "D2Q37":
        c = W.thermal_decay(nx=96, ny=80, tau_hat=0.7, Pr=0.71)
        c.u = W.fp32(c.u + np.array([0.02, -0.01])[:, None, None])
    else:
        c = W.taylor_green_3d(n=24, tau_hat=0.7, Ma=0.1)
        c.params["force"] = False
        c.gfield = None
        c.u = W.fp32(c.u + np.array([0.02, -0.01, 0.015])[:, None, None, None])
    return c


@pytest.mark.parametrize("lattice,storage", [("D2Q37", "f32"), ("D2Q37", "f16"), ("D2Q37", "bf16"),
                                             ("D3Q39", "f32"), ("D3Q39", "f16")])
def test_noalloc_totals_match_diag_on_two_calls(mods, lattice, storage):
    abi, HLBM = mods
    c = _case(lattice)
    D = 2 if lattice == "D2Q37" else 3
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=storage)
    g.init(c.rho, c.u, c.theta)
    g.step(10)                 # even step count: the state is the first buffer of the bound arena
    state = C.c_void_p(g._arena.data_ptr())
    stream = C.c_void_p(abi.hlbm_get_stream(g.ctx))
    lat = abi.HLBM_D2Q37 if lattice == "D2Q37" else abi.HLBM_D3Q39
    st_code = {"f32": abi.HLBM_F32, "f16": abi.HLBM_F16, "bf16": abi.HLBM_BF16}[storage]
    for call in range(2):
        ref = g.diag()         # synchronises the context's stream
        out = (C.c_double * 5)()
        st = abi.hlbm_population_sums_noalloc(lat, c.nodes, st_code, c.params["rho0"], state, stream, out)
        assert st == abi.HLBM_OK
        got = np.array(out[:D + 2])
        mom = np.abs(ref[1:1 + D])
        assert mom.min() > 1e-3 * ref[0]           # a state with net momentum on every axis
        assert abs(got[0] - ref[0]) < 1e-6 * ref[0], (call, got, ref)
        assert np.all(np.abs(got[1:1 + D] - ref[1:1 + D]) < 1e-6 * mom), (call, got, ref)
        assert abs(got[1 + D] - ref[1 + D]) < 1e-6 * ref[1 + D], (call, got, ref)
        g.step(2)
    g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(mods):
    abi, _ = mods
    out = (C.c_double * 5)()
    too_many = 33554432 + 1
    st = abi.hlbm_population_sums_noalloc(abi.HLBM_D2Q37, too_many, abi.HLBM_F32, 1.0, C.c_void_p(16), None, out)
    assert st == abi.HLBM_EINVAL
