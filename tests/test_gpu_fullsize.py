"""GPU parity at the benchmarked sizes, in the launch configurations that are
timed there, against the FP64 oracle.

The persistent kernels hand each resident CTA several tiles in a row and
stage the next tile while the current one collides; that path only runs when
a domain has more tiles than resident CTAs (3 per SM, 456 on GB300).  Every
case here has several tiles per CTA:

* D2Q37 thermal decay 1024^2 (the benchmark workload; 4,096 tiles of 32 x 8)
  on the persistent schedule and on whatever schedule the autotuner picks for
  the benchmark, 100 steps, bar 1e-5 per field (Eq. 4.4; the 1e-5 reading of
  the parity bar);
* the 512^2 van der Waals droplet on the persistent schedule (1,024 tiles);
* the D3Q39 whole-row kernel at 64^3 with a full acceleration field (1,024 row
  tiles);
* the D3Q39 whole-row reverse (adjoint) kernel on a 64 x 64 x 48 box (768
  tiles) against the FP64 reverse-mode oracle;
* at 128^3, T = 400: a checkpoint every 50 steps (recomputed segments) gives
  the same gradient, bit for bit, as keeping every state.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, lattice
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


def _gpu_run(HLBM, c, steps, sched, storage="f32"):
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=storage)
    if sched is not None:
        g.set_tile(*sched)
    if c.gfield is not None:
        g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    g.step(steps)
    m = g.moments_host()
    g.close()
    return m


def _oracle_run(c, steps):
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    if c.gfield is not None:
        o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    o.run(steps)
    return o.moments()


@pytest.fixture(scope="module")
def thermal1024():
    c = W.thermal_decay(n=1024)
    return c, _oracle_run(c, 100)


@pytest.mark.parametrize("sched", [(8, 2, 2), (8, 1, 2), "tuned"])
def test_thermal_1024_benchmark_schedules(HLBM, thermal1024, sched):
    c, mo = thermal1024
    if sched == "tuned":
        from paper_2411_10751_gb300 import autotune
        sched = autotune.tune(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, c.rho, c.u, c.theta)
    mg = _gpu_run(HLBM, c, 100, sched)
    assert max(rel_err(mg, mo)) < TOL32, (sched, rel_err(mg, mo))


@pytest.mark.parametrize("sched", [(8, 1, 2), (8, 2, 2)])
def test_droplet_512_persistent(HLBM, sched):
    c = W.droplet(n=512)
    mg = _gpu_run(HLBM, c, 100, sched)
    mo = _oracle_run(c, 100)
    assert max(rel_err(mg, mo)) < TOL32, (sched, rel_err(mg, mo))


def test_d3q39_rows_kernel_64cube_force_field(HLBM):
    c = W.taylor_green_3d(n=64, tau_hat=0.6, Ma=0.3)
    rng = np.random.default_rng(17)
    c.gfield = W.fp32(2e-5 * (2 * rng.random(c.gfield.shape) - 1))
    mg = _gpu_run(HLBM, c, 40, (8, 2, 2))
    mo = _oracle_run(c, 40)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


def test_adjoint_rows_kernel_many_tiles(HLBM):
    """64 x 64 x 48: 768 whole-row tiles of 4 rows for the reverse kernel."""
    c = W.taylor_green_3d(n=64, tau_hat=0.6, Ma=0.1)
    sl = (slice(0, 48), slice(None), slice(None))
    c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
    c.u = c.u[(slice(None),) + sl].copy()
    c.nz, c.ny, c.nx = c.rho.shape
    rng = np.random.default_rng(23)
    c.gfield = W.fp32(2e-4 * (2 * rng.random((3,) + c.rho.shape) - 1))
    steps, K = 8, 3
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    g.set_tile(8, 2, 2)
    g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    loss, grad = g.adjoint(steps, K)
    grad = grad.cpu().numpy()
    g.close()
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    lref, gref = adjoint.kinetic_energy_gradient(lattice.get(c.lattice), c.rho.shape, c.tau_hat, o.f,
                                                 c.gfield, steps)
    assert abs(loss - lref) < 1e-5 * abs(lref), (loss, lref)
    err = np.abs(grad - gref).max() / np.abs(gref).max()
    assert err < 1e-4, err


def test_adjoint_128_checkpointed_equals_every_state_kept(HLBM):
    """The benchmark's adjoint configuration (128^3, T = 400, a checkpoint every
    50 steps) against the run that keeps all 400 states: recomputation is the
    same kernels on the same inputs, so the gradient agrees bit for bit."""
    import torch
    c = W.taylor_green_3d(n=128, tau_hat=0.6, Ma=0.3, steps=400)
    res = []
    for K in (50, 1):
        g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
        g.set_tile(8, 2, 2)
        g.set_force_field(c.gfield, "field")
        g.init(c.rho, c.u, c.theta)
        loss, grad = g.adjoint(400, K)
        res.append((loss, grad.cpu().numpy()))
        g.close()
        torch.cuda.empty_cache()
    assert res[0][0] == res[1][0]
    assert np.isfinite(res[0][1]).all()
    assert np.array_equal(res[0][1], res[1][1])
