"""GPU adjoint (hlbm_adjoint_run) against the FP64 adjoint oracle.

dL/dg for L = sum rho |u|^2 / 2 after T steps, FP32 on the GPU vs the
torch/FP64 reverse-mode oracle (itself pinned to the C oracle and to finite
differences): max |dg_gpu - dg_ref| / max |dg_ref| < 1e-4.  At the full
128^3 D3Q39 Taylor-Green size the check is a directional finite difference
of the GPU's own forward run (< 1e-2).
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, lattice
from oracle.solver import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def HLBM():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300.solver import HLBM as cls
    return cls


def _case3d(n=16, nx=None, ny=None, nz=None, Ma=0.1, amp=2e-4, seed=5):
    c = W.taylor_green_3d(n=n, tau_hat=0.6, Ma=Ma)
    if nx:
        sl = (slice(0, nz), slice(0, ny), slice(0, nx))
        c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
        c.u = c.u[(slice(None),) + sl].copy()
        c.nz, c.ny, c.nx = c.rho.shape
    rng = np.random.default_rng(seed)
    c.gfield = W.fp32(amp * (2 * rng.random((3,) + c.rho.shape) - 1))
    return c


def _case2d(nx=40, ny=33, seed=6):
    c = W.thermal_decay(nx=nx, ny=ny, tau_hat=0.7, H=False, eps_T=0.02, u0=0.03)
    c.params["force"] = True
    rng = np.random.default_rng(seed)
    c.gfield = W.fp32(2e-4 * (2 * rng.random((2, ny, nx)) - 1))
    return c


def _gpu(HLBM, c, steps, K):
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    loss, grad = g.adjoint(steps, K)
    out = grad.cpu().numpy()
    g.close()
    return loss, out


def _ref(c, steps):
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    L = lattice.get(c.lattice)
    return adjoint.kinetic_energy_gradient(L, c.rho.shape, c.tau_hat, o.f, c.gfield, steps)


@pytest.mark.parametrize("which", ["d3q39_16", "d3q39_ragged", "d3q39_rows32", "d3q39_rows64", "d2q37"])
def test_adjoint_matches_oracle(HLBM, which):
    """d3q39_rows32/64: the whole-row reverse kernel (nx 32 and 64) on ragged
    y (a last tile with rows past the edge, planes copied row by row)."""
    if which == "d3q39_16":
        c, steps, K = _case3d(), 20, 6
    elif which == "d3q39_ragged":
        c, steps, K = _case3d(n=24, nx=21, ny=11, nz=9), 16, 5
    elif which == "d3q39_rows32":
        c, steps, K = _case3d(n=32, nx=32, ny=11, nz=9), 12, 5
    elif which == "d3q39_rows64":
        c, steps, K = _case3d(n=64, nx=64, ny=10, nz=7), 8, 3
    else:
        c, steps, K = _case2d(), 30, 7
    loss, grad = _gpu(HLBM, c, steps, K)
    lref, gref = _ref(c, steps)
    assert abs(loss - lref) < 1e-5 * abs(lref), (loss, lref)
    err = np.abs(grad - gref).max() / np.abs(gref).max()
    assert err < 1e-4, err


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_storage_adjoint(HLBM, storage):
    """16-bit stored forward states (whole-row reverse kernel at nx = 64): the
    gradient stays within the storage rounding of the FP64 one."""
    c, steps, K = _case3d(n=64, nx=64, ny=10, nz=7), 8, 3
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=storage)
    g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    loss, grad = g.adjoint(steps, K)
    grad = grad.cpu().numpy()
    g.close()
    lref, gref = _ref(c, steps)
    err = np.abs(grad - gref).max() / np.abs(gref).max()
    print(storage, "adjoint rel err", err, abs(loss - lref) / abs(lref))
    assert err < 5e-2, err


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_keep_every_state_short_runs(HLBM, steps):
    """Checkpoint interval 1 keeps every state, with the first and last slots
    being the context's own buffers: the shortest runs against the oracle."""
    c = _case3d(n=32, nx=32, ny=11, nz=9)
    loss, grad = _gpu(HLBM, c, steps, 1)
    lref, gref = _ref(c, steps)
    assert abs(loss - lref) < 1e-5 * abs(lref), (loss, lref)
    assert np.abs(grad - gref).max() / np.abs(gref).max() < 1e-4


def test_checkpoint_interval_does_not_change_the_gradient(HLBM):
    c = _case3d()
    res = [_gpu(HLBM, c, 24, K) for K in (1, 5, 24)]
    for loss, grad in res[1:]:
        assert loss == res[0][0]
        assert np.array_equal(grad, res[0][1])


def test_autograd_function(HLBM):
    import torch
    from paper_2411_10751_gb300.solver import KineticEnergy
    c = _case3d()
    solver = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    g = torch.tensor(c.gfield, dtype=torch.float32, device="cuda", requires_grad=True)
    L = KineticEnergy.apply(g, solver, c.rho, c.u, c.theta, 20, 6)
    (dg,) = torch.autograd.grad(2.0 * L, g)
    loss, grad = _gpu(HLBM, c, 20, 6)
    assert abs(L.item() - loss) <= 1e-9 * abs(loss)
    assert np.allclose(dg.cpu().numpy(), 2.0 * grad, rtol=0, atol=1e-7 * np.abs(grad).max())
    solver.close()


def test_full_size_taylor_green_directional_derivative(HLBM):
    """128^3 D3Q39 Taylor-Green (Ma 0.3, tau^ 0.6), T = 400, checkpoint every 50,
    nominal force field 0: <dL/dg, v> against (L(eps v) - L(-eps v)) / (2 eps)."""
    import torch
    c = W.taylor_green_3d(n=128, tau_hat=0.6, Ma=0.3, steps=400)
    loss, grad = _gpu(HLBM, c, 400, 50)
    assert np.isfinite(grad).all() and np.isfinite(loss)
    rng = np.random.default_rng(11)
    v = (2 * rng.random(c.gfield.shape) - 1).astype(np.float32)
    eps = 1e-4

    def ke(gfield):
        g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
        g.set_force_field(gfield, "field")
        g.init(c.rho, c.u, c.theta)
        g.step(400)
        rho, u, _ = g.moments()
        val = 0.5 * (rho.double() * (u.double() ** 2).sum(0)).sum().item()
        g.close()
        return val

    fd = (ke(eps * v) - ke(-eps * v)) / (2 * eps)
    ad = float((grad.astype(np.float64) * v).sum())
    assert abs(fd - ad) < 1e-2 * abs(ad), (fd, ad)
