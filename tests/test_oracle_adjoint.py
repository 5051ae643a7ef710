"""Pins of the FP64 adjoint oracle (P10, no GPU).

1. The torch restatement of the step equals the C oracle's step to round-off
   (two independent codings of the literal Table 2 polynomials).
2. Its reverse-mode gradient of L = sum rho |u|^2 / 2 with respect to the
   force field equals central finite differences of the C oracle's L.
"""
import numpy as np
import pytest

from oracle import adjoint, lattice
from oracle.solver import Oracle
import workloads as W


def _case(name):
    if name == "D3Q39":
        c = W.taylor_green_3d(n=8, tau_hat=0.6, Ma=0.1)
        rng = np.random.default_rng(3)
        g = 2e-4 * (2 * rng.random((3, 8, 8, 8)) - 1)
        return c, g, c.rho.shape
    c = W.thermal_decay(nx=12, ny=9, tau_hat=0.7, Pr=1.0, H=False, eps_T=0.02, u0=0.03)
    c.params["force"] = True
    rng = np.random.default_rng(4)
    g = 2e-4 * (2 * rng.random((2, 9, 12)) - 1)
    return c, g, c.rho.shape


def _oracle(c, g):
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    o.set_force_field(g)
    o.init(c.rho, c.u, c.theta)
    return o


@pytest.mark.parametrize("name", ["D2Q37", "D3Q39"])
def test_torch_step_equals_c_oracle(name):
    import torch
    c, g, shape = _case(name)
    o = _oracle(c, g)
    L = lattice.get(name)
    ts = adjoint.TorchStep(L, shape, c.tau_hat)
    f = torch.tensor(o.f.reshape((L.Q,) + shape))
    gt = torch.tensor(g)
    for _ in range(3):
        f = ts.step(f, gt)
        o.run(1)
        assert np.abs(f.numpy().reshape(L.Q, -1) - o.f).max() < 1e-13 * np.abs(o.f).max()


def _ke(o):
    rho, u, _ = o.moments()
    return 0.5 * float((rho * (u * u).sum(0)).sum())


@pytest.mark.parametrize("name,steps", [("D2Q37", 15), ("D3Q39", 10)])
def test_adjoint_gradient_matches_finite_differences(name, steps):
    c, g, shape = _case(name)
    o = _oracle(c, g)
    L = lattice.get(name)
    loss, dg = adjoint.kinetic_energy_gradient(L, shape, c.tau_hat, o.f, g, steps)
    o.run(steps)
    assert abs(loss - _ke(o)) < 1e-12 * abs(loss)
    rng = np.random.default_rng(9)
    eps = 1e-6
    flat = dg.reshape(-1)
    for idx in rng.choice(flat.size, 6, replace=False):
        gp, gm = g.copy().reshape(-1), g.copy().reshape(-1)
        gp[idx] += eps
        gm[idx] -= eps
        vals = []
        for gg in (gp, gm):
            oo = _oracle(c, gg.reshape(g.shape))
            oo.run(steps)
            vals.append(_ke(oo))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - flat[idx]) <= 1e-6 * max(abs(flat[idx]), 1e-3 * np.abs(flat).max()), (idx, fd, flat[idx])
