"""Physics pins of the FP64 oracle's D3Q39 step (no GPU).

The D3Q39 lattice is not in the paper; its step is the paper's method
(Eqs. 4.4-4.5 with the equilibrium of Eq. 2.2 truncated after the third
order and the body force of Eq. 3.3) on the degree-7 three-dimensional
lattice.  These tests fix that step by physics, each chosen so that a
plausible slip in the oracle's 3D code fails one of them:

* conservation in a periodic box (Eq. 2.3; the collision keeps the moments
  rho, rho u and the energy): mass, momentum and energy constant to round-off
  over 500 steps.  A wrong dimension in the temperature of Eq. 4.5 (the
  rho D c0^2 denominator) breaks the energy.
* a uniform acceleration raises the momentum by exactly g * mass per step
  (s^(1) = F, Eq. 3.2, and the half-force shift of Eq. 4.5).
* a shear wave along each axis, in a frame moving along the wave vector,
  decays at nu k^2 with nu = c0^2 (tau^ - 1/2) and is carried at the frame's
  speed.  The wave along z fails for a mis-signed z wrap; the moving frame
  (Galilean invariance of the stress) needs the third-order terms of
  Eq. 2.2.
* the entropy mode (temperature wave at constant pressure) decays at
  (nu / Pr) k^2: Pr = 1 for BGK alone (Sec. 1) and the Pr of the thermal
  source H_i (Eqs. 3.4-3.7) with it.
* the Taylor-Green vortex's kinetic energy decays at first at 6 nu k^2
  (three Fourier components with |k|^2 = 3 (2 pi / n)^2).
* the oracle's whole step equals a brute-force Hermite-tensor step (Eqs. 2.4-
  2.6, 3.2, 3.6, 4.4-4.5 from full Cartesian tensors) on a 7 x 7 x 7 box.
"""
import numpy as np
import pytest

import workloads as W
from oracle import analytic, lattice
from oracle.solver import Oracle

from test_oracle_bruteforce import brute_step


def _smooth3d(nx, ny, nz, amp=0.02):
    z, y, x = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    rho = 1.0 + amp * np.sin(x) * np.cos(2 * y) * np.cos(z)
    u = np.stack([amp * np.cos(y + z), amp * np.sin(2 * x - z), amp * np.cos(x + y)])
    theta = 1.0 + amp * np.cos(x - y + 2 * z)
    return rho, u, theta


def test_d3q39_conservation_periodic_box():
    rho, u, th = _smooth3d(14, 12, 10)
    o = Oracle("D3Q39", 14, 12, 10, 0.7, W.source_params())
    o.init(rho, u, th)
    d0 = o.diag()
    o.run(500)
    d1 = o.diag()
    M, E = d0[0], d0[4]
    assert abs(d1[0] - M) <= 1e-12 * M
    assert np.all(np.abs(d1[1:4] - d0[1:4]) <= 1e-12 * M)
    assert abs(d1[4] - E) <= 1e-12 * E
    # the state did evolve: the energy exchange between modes is not trivial
    assert np.abs(o.moments()[1] - u).max() > 1e-3


def test_d3q39_conservation_with_thermal_source():
    """H_i has zero 0th, 1st and 2nd moments (only s^(3) is non-zero, Eq. 3.6)."""
    rho, u, th = _smooth3d(10, 9, 8)
    o = Oracle("D3Q39", 10, 9, 8, 0.65, W.source_params(H=True, Pr=0.71))
    o.init(rho, u, th)
    d0 = o.diag()
    o.run(300)
    d1 = o.diag()
    assert abs(d1[0] - d0[0]) <= 1e-12 * d0[0]
    assert np.all(np.abs(d1[1:4] - d0[1:4]) <= 1e-12 * d0[0])
    assert abs(d1[4] - d0[4]) <= 1e-12 * d0[4]


def test_d3q39_uniform_force_momentum_budget():
    rho, u, th = _smooth3d(12, 10, 9)
    g = (2e-5, -1e-5, 3e-5)
    o = Oracle("D3Q39", 12, 10, 9, 0.9, W.source_params(force=True, g=g))
    o.init(rho, u, th)
    d0 = o.diag()
    o.run(50)
    d1 = o.diag()
    assert abs(d1[0] - d0[0]) <= 1e-12 * d0[0]
    assert np.allclose(d1[1:4] - d0[1:4], 50 * d0[0] * np.array(g), rtol=1e-10, atol=1e-14)


def _wave_box(axis, n):
    shape = [1, 1, 1]                 # (nz, ny, nx)
    shape[2 - axis] = n
    return tuple(shape)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("tau_hat,U0", [(0.8, 0.0), (0.8, 0.2), (0.6, 0.3)])
def test_d3q39_shear_wave_galilean(axis, tau_hat, U0):
    """u_t = u0 sin(k s) along axis `axis` (s its coordinate, t the next axis),
    plus a uniform velocity U0 along the wave vector.  Fields that vary along
    one axis only: the other two extents are 1, which is exact for such states
    (every neighbour along them is the node itself)."""
    n = 64
    shape = _wave_box(axis, n)
    s = np.arange(n)
    k = 2 * np.pi / n
    t = (axis + 1) % 3
    prof = 1e-4 * np.sin(k * s)
    u = np.zeros((3,) + shape)
    u[t] = prof.reshape(shape)
    u[axis] = U0
    nz, ny, nx = shape
    o = Oracle("D3Q39", nx, ny, nz, tau_hat, W.source_params())
    o.init(np.ones(shape), u, np.ones(shape))

    def amp():
        ut = o.moments()[1][t].reshape(n)
        return (ut * np.exp(-1j * k * s)).sum() * 2 / n

    o.run(50)
    a0 = a = amp()
    phase = 0.0
    for _ in range(100):
        o.run(10)
        b = amp()
        phase += -np.angle(b / a)
        a = b
    nu = analytic.viscosity(lattice.d3q39().cs2, tau_hat)
    rate = np.log(abs(a0) / abs(a)) / 1000
    assert abs(rate / (nu * k * k) - 1) < 5e-3, rate / (nu * k * k)
    assert abs(phase / (k * 1000) - U0) < 1e-3 * max(U0, 0.1), phase / (k * 1000)


def _entropy_rate_3d(Pr, H, n=64, tau_hat=0.7, axis=2):
    shape = _wave_box(axis, n)
    s = np.arange(n)
    sn = np.sin(2 * np.pi * s / n)
    theta = (1.0 + 1e-4 * sn).reshape(shape)
    nz, ny, nx = shape
    o = Oracle("D3Q39", nx, ny, nz, tau_hat, W.source_params(H=H, Pr=Pr))
    o.init(1.0 / theta, np.zeros((3,) + shape), theta)
    nu = analytic.viscosity(lattice.d3q39().cs2, tau_hat)
    expect = analytic.entropy_mode_rate(nu, Pr, n)
    o.run(int(0.2 / expect))
    ts, am = [], []
    T1 = int(1.0 / expect)
    stride = max(1, T1 // 200)
    for t in range(0, T1, stride):
        th = o.moments()[2].reshape(n)
        ts.append(t)
        am.append(((th - 1.0) * sn).sum() / (sn * sn).sum())
        o.run(stride)
    # least squares over many acoustic periods (sound waves ride on the decay)
    return -np.polyfit(ts, np.log(am), 1)[0], expect


@pytest.mark.parametrize("Pr,H,axis", [(1.0, False, 2), (1.0, False, 0), (0.71, True, 2), (1.41, True, 1)])
def test_d3q39_entropy_mode_prandtl(Pr, H, axis):
    rate, expect = _entropy_rate_3d(Pr, H, axis=axis)
    assert abs(rate / expect - 1) < 1e-2, (rate, expect)


def test_d3q39_taylor_green_early_decay():
    """P11: the Taylor-Green vortex at 32^3 loses kinetic energy at 6 nu k^2
    (k = 2 pi / 32) over its first 40 steps, within 2%.  Ma 0.05: the energy
    cascade to higher wavenumbers raises the dissipation with the Reynolds
    number (at Ma 0.1 and tau^ 0.6 the rate is already 4% higher)."""
    n, tau_hat = 32, 0.8
    c = W.taylor_green_3d(n=n, tau_hat=tau_hat, Ma=0.05)
    p = dict(c.params)
    p["force"] = False
    o = Oracle("D3Q39", n, n, n, tau_hat, p)
    o.init(c.rho, c.u, c.theta)

    def ke():
        r, u, _ = o.moments()
        return 0.5 * (r * (u * u).sum(0)).sum()

    ks = [ke()]
    for _ in range(40):
        o.run(1)
        ks.append(ke())
    rate = -np.polyfit(np.arange(41), np.log(ks), 1)[0]
    nu = analytic.viscosity(lattice.d3q39().cs2, tau_hat)
    k = 2 * np.pi / n
    assert abs(rate / (6 * nu * k * k) - 1) < 2e-2, rate / (6 * nu * k * k)


@pytest.mark.parametrize("case", ["force_field", "force_H"])
def test_d3q39_oracle_step_equals_hermite_tensor_step(case):
    """The oracle's literal polynomials against the general Hermite-tensor
    expansion on 7 x 7 x 7 (third-order equilibrium, Eq. 2.2 truncated), 2 steps."""
    L = lattice.d3q39()
    shape = (7, 7, 7)
    rng = np.random.default_rng(21)
    g = 1e-3 * (2 * rng.random((3,) + shape) - 1)
    p = W.source_params(force=True, H=(case == "force_H"), Pr=0.71)
    fld = W.random_small("D3Q39", nx=7, ny=7, nz=7, seed=8)
    o = Oracle("D3Q39", 7, 7, 7, 0.71, p)
    o.init(fld["rho"], fld["u"], fld["theta"])
    o.f += 1e-3 * L.w[:, None] * (2 * rng.random(o.f.shape) - 1)
    o.set_force_field(g)
    f = o.f.copy()
    for _ in range(2):
        f = brute_step(L, p, 0.71, f, g, shape)
        o.run(1)
        assert np.abs(o.f - f).max() < 1e-13 * np.abs(f).max(), np.abs(o.f - f).max()
