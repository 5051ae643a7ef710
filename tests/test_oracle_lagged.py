"""Physics pins of the oracle's single-pass variant (neighbour fields of the
previous step), on which the in-place (AA-pattern) GPU step is checked.

In the single-pass variant grad theta (H_i, Eq. 3.7) and the pseudopotential
field of F^SC and P_i (Eqs. 3.8, 3.12) come from the previous step's
temperature and density; everything else is Eq. 4.4 at time t.  It changes
results, so it is re-validated here against the same physics as the exact
two-pass scheme (P5-P9):

* with neither source the two schemes are identical;
* conservation: mass, momentum and energy with H_i, mass and momentum with
  F^SC + P_i (the lagged F^SC is still pairwise antisymmetric);
* the Prandtl number the thermal source sets (entropy-mode decay);
* liquid-gas coexistence: a flat interface settles to the same bulk densities
  (in a steady state the previous step's fields are this step's).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import analytic, lattice
from oracle.solver import Oracle

from test_oracle_physics import _smooth_fields


def _lagged(params, lag=True):
    p = dict(params)
    p["lag"] = lag
    return p


def test_without_neighbour_fields_the_variants_are_identical():
    c = W.kolmogorov(nx=24, ny=20)
    out = []
    for lag in (False, True):
        o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, _lagged(c.params, lag))
        o.set_force_field(c.gfield)
        o.init(c.rho, c.u, c.theta)
        o.run(50)
        out.append(o.f.copy())
    assert np.array_equal(out[0], out[1])


def test_lagged_conservation_thermal_source():
    rho, u, th = _smooth_fields(16, 16)
    o = Oracle("D2Q37", 16, 16, 1, 0.7, _lagged(W.source_params(H=True, Pr=0.71)))
    o.init(rho, u, th)
    d0 = o.diag()
    o.run(1000)
    d1 = o.diag()
    assert abs(d1[0] - d0[0]) <= 1e-12 * d0[0]
    assert np.all(np.abs(d1[1:3] - d0[1:3]) <= 1e-12 * d0[0])
    assert abs(d1[3] - d0[3]) <= 1e-12 * d0[3]


def test_lagged_conservation_pseudopotential():
    c = W.droplet(n=32, r0=8.0, tau_hat=0.8, k=1.0)
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, _lagged(c.params))
    o.init(c.rho, c.u, c.theta)
    d0 = o.diag()
    o.run(300)
    d1 = o.diag()
    assert np.isfinite(d1).all()
    assert abs(d1[0] - d0[0]) <= 1e-12 * d0[0]
    assert np.all(np.abs(d1[1:3] - d0[1:3]) <= 1e-12 * d0[0])


@pytest.mark.parametrize("Pr", [0.71, 1.41])
def test_lagged_prandtl_number(Pr):
    nx, tau_hat = 128, 0.7
    c = W.thermal_decay(nx=nx, ny=8, tau_hat=tau_hat, Pr=Pr, noise=0, u0=0.0, eps_T=1e-4, H=True)
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, _lagged(c.params))
    o.init(c.rho, c.u, c.theta)
    s = np.sin(2 * np.pi * np.arange(nx) / nx)
    nu = analytic.viscosity(o.L.cs2, tau_hat)
    k2 = analytic.entropy_mode_rate(nu, Pr, nx)
    o.run(int(0.2 / k2))
    ts, am = [], []
    T1 = int(1.0 / k2)
    stride = max(1, T1 // 200)
    for t in range(0, T1, stride):
        _, _, th = o.moments()
        ts.append(t)
        am.append(((th.mean(axis=0) - 1.0) * s).sum() / (s * s).sum())
        o.run(stride)
    rate = -np.polyfit(ts, np.log(am), 1)[0]
    assert abs(rate / k2 - 1) < 1e-2, (rate, k2)


def test_lagged_flat_interface_matches_maxwell():
    path = os.path.join(os.path.dirname(__file__), "golden", "vdw_flat_interface_k.txt")
    k = float([ln for ln in open(path) if not ln.startswith("#")][0])
    c = W.flat_interface(nx=8, ny=200, tau_hat=0.8, Tr=0.85, k=k, eos="vdw")
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, _lagged(c.params))
    o.init(c.rho, c.u, c.theta)
    o.run(10000)
    rho, _, _ = o.moments()
    assert abs(rho[0, 0] / c.meta["rho_g"] - 1) < 2e-2
    assert abs(rho[100, 0] / c.meta["rho_l"] - 1) < 2e-2
