"""Physics pins of the oracle's wall boundary (Sec. 4.3, Eqs. 4.7-4.8) and of
the wall cases of Sec. 5.1-5.3 (no GPU).

Geometry (the reading of Sec. 5.1's "actual height 54" for 56 rows and of
Sec. 5.3's H = 100 for 102 rows): the wall nodes are rows 0 and ny - 1 and
the solid-liquid interfaces lie half a cell inside them, at y = 1/2 and
y = ny - 3/2, so H = ny - 2.

Flows that vary along y only run on nx = 1 (every x neighbour is the node
itself, exact for x-invariant states; checked against nx = 8 below).
c_p = (D + 2) c0^2 / 2 = 2 c0^2 is the specific heat at constant pressure in
units of theta (Eq. 5.3's Ec = u0^2 / (c_p Delta theta)), pinned in the bulk
by the forced Kolmogorov flow's heating below.

* A fluid at rest at the wall temperature stays at rest, and mass is
  conserved to round-off (impermeable walls).
* Couette (Eq. 5.1): the profile is linear, with u = 0 and u = u0 within a
  quarter cell of the interfaces; as printed, Eq. 4.7 passes almost none of
  the wall's momentum into the fluid.
* Conduction between walls at different temperatures: theta is linear and
  takes the wall temperatures within a quarter cell of the interfaces, with
  and without the thermal source (Pr 0.71, 1, 1.41).
* Couette heating (Eq. 5.2): in the bulk theta'' = -(Pr / c_p) u'^2, and the
  whole theta* profile follows Eq. 5.2 with the simulated shear.
* Poiseuille (Eq. 5.4): u'' = -g / nu; its heating (Eq. 5.5) follows
  theta'' = -(Pr / c_p) u'^2.
* Rayleigh-Benard (Sec. 5.3): rest is stable below the rigid-rigid critical
  Rayleigh number 1707.8 and unstable above it (Ra taken with the viscosity
  and diffusivity at the mean temperature).
"""
import numpy as np
import pytest

import workloads as W
from oracle import lattice, solver
from oracle.solver import Oracle

L = lattice.d2q37()
CP = 2.0 * L.cs2


def _run_1d(ny, tau, steps, **kw):
    th0 = kw.pop("theta0", 1.0)
    p = W.source_params(walls=True, **kw)
    o = Oracle("D2Q37", 1, ny, 1, tau, p)
    o.init(np.full((ny, 1), 1.0 / th0), np.zeros((2, ny, 1)), np.full((ny, 1), th0))
    threads = solver.get_threads()
    solver.set_threads(1)            # a column of a few dozen nodes: threads cost more than they give
    try:
        o.run(steps)
    finally:
        solver.set_threads(threads)
    r, u, t = o.moments()
    return r[:, 0], u[0][:, 0], u[1][:, 0], t[:, 0], o


def test_tabulated_lattice_constant():
    assert W.CS2_D2Q37 == L.cs2


def test_rest_state_at_wall_temperature_is_kept():
    ny, nx = 16, 4
    p = W.source_params(walls=True, wall_theta=(1.1, 1.1), H=True, Pr=0.71)
    o = Oracle("D2Q37", nx, ny, 1, 0.7, p)
    o.init(np.full((ny, nx), 0.9), np.zeros((2, ny, nx)), np.full((ny, nx), 1.1))
    o.run(200)
    r, u, t = o.moments()
    assert np.abs(r - 0.9).max() < 1e-12 and np.abs(u).max() < 1e-13 and np.abs(t - 1.1).max() < 1e-12


def test_x_invariant_states_do_not_depend_on_nx():
    res = []
    for nx in (1, 8):
        p = W.source_params(walls=True, wall_u=((0, 0, 0), (0.03, 0, 0)), wall_theta=(1.0, 1.02), H=True, Pr=0.71,
                            force=True, g=(1e-5, 0, 0))
        o = Oracle("D2Q37", nx, 20, 1, 0.7, p)
        o.init(np.ones((20, nx)), np.zeros((2, 20, nx)), np.ones((20, nx)))
        o.run(300)
        res.append(o.moments())
    for a, b in zip(*res):
        assert np.array_equal(a[..., :1], b[..., :1]) and np.all(b == b[..., :1])


def test_walls_conserve_mass():
    c = W.rayleigh_benard(nx=24, ny=18, Ra=5000.0)
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    o.init(c.rho, c.u, c.theta)
    m0 = o.moments()[0].sum()
    o.run(1000)
    r, u, _ = o.moments()
    assert np.isfinite(r).all()
    assert abs(r.sum() - m0) < 1e-12 * m0


def _line(y, v):
    a, b = np.polyfit(y, v, 1)
    return a, b, np.abs(v - (a * y + b)).max()


@pytest.mark.parametrize("tau", [0.55, 0.7, 1.0])
def test_couette_linear_profile(tau):
    ny, u0 = (16 if tau < 0.6 else 24), 0.02
    nu = L.cs2 * (tau - 0.5)
    _, ux, uy, _, _ = _run_1d(ny, tau, int(12 * ny * ny / nu), wall_u=((0, 0, 0), (u0, 0, 0)))
    y = np.arange(ny)
    a, b, res = _line(y[3:-3], ux[3:-3])
    assert res < 5e-3 * u0                                        # Eq. 5.1: linear
    lo, hi = -b / a, (u0 - b) / a                                 # where u = 0 and u = u0
    assert abs(lo - 0.5) < 0.25 and abs(hi - (ny - 1.5)) < 0.25, (lo, hi)
    assert np.abs(uy).max() < 1e-5 * 100 * u0


def test_couette_printed_rule_is_rejected():
    ny, u0, tau = 24, 0.02, 0.8
    _, ux, _, _, _ = _run_1d(ny, tau, 20000, wall_u=((0, 0, 0), (u0, 0, 0)), wall_rule=1)
    a, _, _ = _line(np.arange(3, ny - 3), ux[3:-3])
    assert a < 0.3 * u0 / (ny - 2)


@pytest.mark.parametrize("tau,Pr,H", [(0.56, 1.0, False), (0.56, 0.71, True), (0.56, 1.41, True),
                                      (0.8, 1.0, False), (0.8, 0.71, True)])
def test_conduction_wall_temperatures(tau, Pr, H):
    ny, tb, tt = (16 if tau < 0.6 else 24), 1.0, 1.01
    nu = L.cs2 * 1.005 * (tau - 0.5)
    _, _, _, th, _ = _run_1d(ny, tau, int(10 * ny * ny * max(Pr, 1.0) / nu), wall_theta=(tb, tt), H=H, Pr=Pr,
                             theta0=0.5 * (tb + tt))
    y = np.arange(ny)
    a, b, res = _line(y[3:-3], th[3:-3])
    assert res < 1e-2 * (tt - tb)
    lo, hi = (tb - b) / a, (tt - b) / a
    assert abs(lo - 0.5) < 0.25 and abs(hi - (ny - 1.5)) < 0.25, (lo, hi)


def test_kolmogorov_viscous_heating_sets_c_p():
    """Periodic forced flow u = U sin(k y): the dissipation mu U^2 k^2 cos^2(k y)
    balances conduction in the cos(2 k y) temperature mode, whose amplitude is
    Pr U^2 / (8 c_p) with c_p = 2 c0^2 (D = 2), for BGK (Pr = 1) and with H_i."""
    n, tau = 64, 0.8
    k = 2 * np.pi / n
    nu = L.cs2 * (tau - 0.5)
    U = 0.05
    y = np.arange(n)
    for Pr, H in ((1.0, False), (0.71, True), (1.41, True)):
        gf = np.zeros((2, n, 1))
        gf[0] = (U * nu * k * k * np.sin(k * y))[:, None]
        o = Oracle("D2Q37", 1, n, 1, tau, W.source_params(force=True, H=H, Pr=Pr))
        o.set_force_field(gf)
        u0 = np.zeros((2, n, 1))
        u0[0] = (U * np.sin(k * y))[:, None]
        o.init(np.ones((n, 1)), u0, np.ones((n, 1)))
        o.run(3000)
        _, u, t = o.moments()
        Um = (u[0][:, 0] * np.sin(k * y)).sum() * 2 / n
        th2 = (t[:, 0] * np.cos(2 * k * y)).sum() * 2 / n
        assert abs(th2 / (Pr * Um * Um / (8 * CP)) - 1) < 1e-2, (Pr, th2)


def _second_derivative(v):
    return v[2:] - 2 * v[1:-1] + v[:-2]


@pytest.mark.parametrize("Pr,H", [(1.0, False), (0.71, True), (1.41, True)])
def test_couette_viscous_heating_eq_5_2(Pr, H):
    """Eq. 5.2 with both walls at one temperature: theta - theta_w =
    Pr u'^2 H^2 / (2 c_p) y*(1 - y*).  In the bulk the curvature is exact
    (kappa theta'' = -mu u'^2).  At the resting wall the fluid takes the wall
    temperature within 0.35 cells of the interface (a Knudsen-layer jump);
    the moving wall (Sec. 5.1's top wall) adds a jump of its own, about
    0.02-0.025 u0^2 / c_p at tau^ = 0.8, whatever Pr."""
    ny, tau, u0 = 24, 0.8, 0.05
    nu = L.cs2 * (tau - 0.5)
    _, ux, _, th, _ = _run_1d(ny, tau, int(15 * ny * ny * max(Pr, 1.0) / nu), wall_u=((0, 0, 0), (u0, 0, 0)),
                              H=H, Pr=Pr)
    y = np.arange(ny)
    du, b, _ = _line(y[4:-4], ux[4:-4])
    c = np.polyfit(y[4:-4], th[4:-4], 2)
    assert abs(2 * c[0] / (-Pr / CP * du * du) - 1) < 2e-2
    rise = Pr * (du * (ny - 2)) ** 2 / (8 * CP)
    slope_wall = 4 * rise / (ny - 2)                      # |theta'| at the interfaces
    jump_rest = np.polyval(c, 0.5) - 1.0
    jump_moving = np.polyval(c, ny - 1.5) - 1.0
    assert 0 <= jump_rest < 0.35 * slope_wall, (jump_rest, slope_wall)
    assert 0 <= jump_moving < 0.03 * u0 * u0 / CP, (jump_moving, u0 * u0 / CP)


def test_poiseuille_profile():
    ny, tau = 24, 0.6
    nu = L.cs2 * (tau - 0.5)
    g = 8 * nu * 0.02 / (ny - 2) ** 2
    _, ux, _, _, _ = _run_1d(ny, tau, int(15 * ny * ny / nu), force=True, g=(g, 0, 0))
    y = np.arange(ny)
    c = np.polyfit(y[2:-2], ux[2:-2], 2)
    assert abs(2 * c[0] / (-g / nu) - 1) < 5e-3                   # Eq. 5.4: u'' = -g / nu
    lo, hi = np.sort(np.roots(c).real)
    assert abs(lo - 0.5) < 0.25 and abs(hi - (ny - 1.5)) < 0.25, (lo, hi)


@pytest.mark.parametrize("Pr,H", [(1.0, False), (0.71, True), (1.41, True)])
def test_poiseuille_heating_eq_5_5(Pr, H):
    """Eq. 5.5's quartic: with u = a y^2 + b y + c, kappa theta'' = -mu u'^2
    makes the y^4 coefficient of theta -(Pr / c_p) a^2 / 3."""
    ny, tau, uc = 40, 0.8, 0.05
    nu = L.cs2 * (tau - 0.5)
    g = 8 * nu * uc / (ny - 2) ** 2
    _, ux, _, th, _ = _run_1d(ny, tau, int(15 * ny * ny * max(Pr, 1.0) / nu), force=True, g=(g, 0, 0), H=H, Pr=Pr)
    y = np.arange(ny)
    a = np.polyfit(y[2:-2], ux[2:-2], 2)[0]
    c4 = np.polyfit(y[3:-3], th[3:-3], 4)[0]
    assert abs(c4 / (-(Pr / CP) * a * a / 3) - 1) < 3e-2, c4 / (-(Pr / CP) * a * a / 3)


def _rb_growth(Ra, H=20):
    c = W.rayleigh_benard(nx=2 * H, ny=H + 2, Ra=Ra)
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    o.init(c.rho, c.u, c.theta)
    xx = np.arange(c.nx)
    amp = []
    for _ in range(6):
        o.run(1500)
        mid = o.moments()[1][1][c.ny // 2]
        amp.append(abs((mid * np.exp(-2j * np.pi * xx / c.nx)).sum()) * 2 / c.nx)
    return np.log(amp[-1] / amp[-3]) / 3000


def test_rayleigh_benard_onset():
    """L = 2H, so the first mode has k = pi / H, close to the critical 3.117 / H.
    Rest decays at 0.85 x 1707.8 and grows at 1.2 x 1707.8 (Ra of Eq. 5.6 with
    the viscosity and expansion coefficient at the mean temperature)."""
    assert _rb_growth(0.85 * 1707.8) < 0
    assert _rb_growth(1.2 * 1707.8) > 0
