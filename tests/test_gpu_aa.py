"""GPU parity of the in-place (AA-pattern) step with single-pass neighbour
fields (HLBM_AA) against the oracle's single-pass variant (FP64), through
the C ABI.

Bar as in test_gpu_parity.py: per field max |q_gpu - q_oracle| / max |q_oracle|
< 1e-5 after 100 steps (FP32 storage).  Odd and even step counts are checked
(the two halves of the AA pattern leave different layouts in memory).
"""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Oracle

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def HLBM():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300.solver import HLBM as cls
    return cls


def rel_err(m_gpu, m_ora):
    rho, u, th = m_gpu
    r0, u0, t0 = m_ora
    er = np.abs(rho - r0).max() / np.abs(r0).max()
    eu = np.sqrt(((u - u0) ** 2).sum(0)).max() / max(np.sqrt((u0 ** 2).sum(0)).max(), 1e-300)
    et = np.abs(th - t0).max() / np.abs(t0).max()
    return er, eu, et


def lagged(c):
    c.params = dict(c.params)
    c.params["lag"] = True
    return c


def _gpu(HLBM, c, steps, storage="f32"):
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params, storage=storage)
    if c.gfield is not None:
        g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    g.step(steps)
    m = g.moments_host()
    g.close()
    return m


def _oracle(c, steps):
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    if c.gfield is not None:
        o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    o.run(steps)
    return o.moments()


@pytest.mark.parametrize("steps", [1, 2, 3, 100, 101])
def test_aa_thermal_parity(HLBM, steps):
    c = lagged(W.thermal_decay(nx=200, ny=120, tau_hat=0.7, Pr=0.71))
    assert max(rel_err(_gpu(HLBM, c, steps), _oracle(c, steps))) < TOL32


@pytest.mark.parametrize("nx,ny", [(7, 7), (45, 37), (96, 64)])
def test_aa_droplet_parity(HLBM, nx, ny):
    """u is compared on the velocity scale max(max|u|, 0.01): a small droplet's
    velocity is its spurious current (0.0033 at 45 x 37), and its liquid is
    stored as deviations of about 5.2 from the gas reference density (FP32 ulp
    4.8e-7, about 1e-7 in u after 100 steps), as in the batched test."""
    c = lagged(W.droplet(nx=nx, ny=ny, r0=0.25 * min(nx, ny), k=1.5672))
    steps = 10 if nx == 7 else 100
    mo = _oracle(c, steps)
    er, eu, et = rel_err(_gpu(HLBM, c, steps), mo)
    umax = np.sqrt((mo[1] ** 2).sum(0)).max()
    eu *= umax / max(umax, 0.01)
    assert max(er, eu, et) < TOL32, (er, eu, et)


def test_aa_body_force_equals_two_buffer_step_bitwise(HLBM):
    """Without neighbour fields the in-place step and the two-buffer step do the
    same arithmetic: equal moments, bit for bit, at odd and even counts."""
    for steps in (7, 40):
        c = W.kolmogorov(nx=64, ny=48)
        a = _gpu(HLBM, lagged(W.kolmogorov(nx=64, ny=48)), steps)
        g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
        g.set_tile(8, 1, 1)
        g.set_force_field(c.gfield, "field")
        g.init(c.rho, c.u, c.theta)
        g.step(steps)
        b = g.moments_host()
        g.close()
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_aa_thermal_1024(HLBM):
    c = lagged(W.thermal_decay(n=1024))
    assert max(rel_err(_gpu(HLBM, c, 100), _oracle(c, 100))) < TOL32


def test_aa_fp16_storage(HLBM):
    c = lagged(W.thermal_decay(nx=256, ny=256, tau_hat=0.7, Pr=0.71))
    er, eu, et = rel_err(_gpu(HLBM, c, 100, storage="f16"), _oracle(c, 100))
    assert eu < 1e-3, (er, eu, et)


def test_aa_graph_replay_save_load_memory(HLBM):
    """70 steps as graph replays equal 70 single steps; a save at an odd step
    count resumes bit for bit; the workspace is about half the two-buffer one."""
    from paper_2411_10751_gb300 import abi, solver
    c = lagged(W.droplet(nx=64, ny=48, r0=12.0, k=1.0))
    g1 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g2 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g1.init(c.rho, c.u, c.theta)
    g2.init(c.rho, c.u, c.theta)
    g1.step(70)
    for _ in range(70):
        g2.step(1)
    for x, y in zip(g1.moments_host(), g2.moments_host()):
        assert np.array_equal(x, y)
    g1.step(5)
    state = g1.save()
    g1.step(20)
    ref = g1.moments_host()
    g3 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g3.load(state)
    assert g3.step_count == 75
    g3.step(20)
    for x, y in zip(ref, g3.moments_host()):
        assert np.array_equal(x, y)
    two = dict(c.params)
    two["lag"] = False
    import ctypes as C
    n_aa = abi.hlbm_workspace_bytes(abi.HLBM_D2Q37, 1024, 1024, 1, C.byref(solver.make_params(c.params)))
    n_two = abi.hlbm_workspace_bytes(abi.HLBM_D2Q37, 1024, 1024, 1, C.byref(solver.make_params(two)))
    assert n_aa < 0.6 * n_two, (n_aa, n_two)
    for g in (g1, g2, g3):
        g.close()
