"""P12: the oracle's whole step against a brute-force Hermite-tensor step.

The oracle evaluates the literal Table 2 polynomials.  This test rebuilds the
same step from the general expansion instead: full Cartesian Hermite tensors
H^(n)(xi) = xi^n - [delta xi^(n-2)] + [delta^2 xi^(n-4)] (Eq. 2.4), the
equilibrium coefficients of Eq. 2.6 (with + theta-bar^2 [delta delta]), the
source coefficients of Eqs. 3.2, 3.6 and 3.12, f = w sum_n a^(n):H^(n) / n!
(Eq. 2.5), then Eqs. 4.4-4.5 and periodic streaming with np.roll, on a 7 x 7
grid (the smallest size where reach-3 velocities do not alias) for 3 steps.
Both routes must agree to round-off.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import eos, lattice
from oracle.solver import Oracle
import workloads as W


def sym(T):
    """Average of T over all permutations of its axes."""
    n = T.ndim
    if n < 2:
        return T
    return sum(np.transpose(T, p) for p in itertools.permutations(range(n))) / math.factorial(n)


def outer(*vs):
    t = np.ones(())
    for v in vs:
        t = np.multiply.outer(t, v)
    return t


def hermite_tensors(xi, D):
    d = np.eye(D)
    H = [np.ones(()), xi.copy(), outer(xi, xi) - d,
         outer(xi, xi, xi) - 3 * sym(outer(d, xi)),
         outer(xi, xi, xi, xi) - 6 * sym(outer(d, xi, xi)) + 3 * sym(outer(d, d))]
    return H


def contract(a, h):
    return float(np.sum(a * h))


def brute_step(L, p, tau_hat, f, g, shape):
    D, Q = L.D, L.Q
    c0, cs2 = L.c0, L.cs2
    d = np.eye(D)
    Ht = [hermite_tensors(L.c[i] / c0, D) for i in range(Q)]
    N = int(np.prod(shape))
    fl = f.reshape(Q, N)
    rho = fl.sum(axis=0)
    isothermal = p.get("isothermal", False)
    psi = np.zeros(N)
    if p.get("SC"):
        pe = eos.pressure(p["eos"], rho, p["eos_a"], p["eos_b"], p["eos_T"])
        psi = np.sqrt(np.maximum(2.0 * (pe - rho * cs2) / (-1.0 * cs2), 0.0))
    psi_g = psi.reshape(shape)

    def shifted(field, cvec):
        # field(x + c): roll by -c along each axis (arrays are [.., y, x])
        axes = tuple(range(field.ndim - 1, -1, -1))[:D]
        return np.roll(field, shift=tuple(-int(cvec[a]) for a in range(D)), axis=axes)

    Fsc = np.zeros((D, N))
    if p.get("SC"):
        acc = np.zeros((D,) + shape)
        for i in range(Q):
            acc += L.w[i] * shifted(psi_g, L.c[i])[None] * L.c[i].reshape((D,) + (1,) * D)
        Fsc = (-(-1.0) * psi_g[None] * acc).reshape(D, N)
    if g is not None:
        gg = g.reshape(D, N)
    elif p.get("force"):
        gg = np.repeat(np.asarray(p["g"][:D], float)[:, None], N, axis=1)
    else:
        gg = np.zeros((D, N))
    F = rho * gg + Fsc
    j = L.c.T.astype(float) @ fl
    u = (j + 0.5 * F) / rho
    tau = tau_hat - 0.5
    sigma = np.zeros(N)
    if p.get("SC") and p.get("P"):
        sigma = np.where(psi > 0, -p["k"] * cs2 * (Fsc * Fsc).sum(0) / (D * tau * -1.0 * np.where(psi > 0, psi, 1.0) ** 2), 0.0)
    cc = (L.c ** 2).sum(axis=1).astype(float)
    # G2 = c0^2 tr s^(2) = 2 u.F + D c0^2 sigma
    G2 = 2.0 * (u * F).sum(0) + D * cs2 * sigma
    theta = (cc @ fl - rho * (u * u).sum(0) + 0.5 * G2) / (rho * D * cs2)
    th = np.ones(N) if isothermal else theta
    gradT = np.zeros((D, N))
    if p.get("H"):
        tg = theta.reshape(shape)
        for a in range(D):
            e = np.zeros(D, dtype=int)
            e[a] = 1
            gradT[a] = (0.5 * (shifted(tg, e) - shifted(tg, -e))).reshape(N)
    fstar = np.zeros_like(fl)
    for n in range(N):
        r, tb = rho[n], th[n] - 1.0
        ux, Fx = u[:, n] / c0, F[:, n] / c0
        a = [r * np.ones(()), r * ux, r * (outer(ux, ux) + tb * d),
             r * (outer(ux, ux, ux) + tb * 3 * sym(outer(ux, d))),
             r * (outer(ux, ux, ux, ux) + tb * 6 * sym(outer(ux, ux, d)) + tb * tb * 3 * sym(outer(d, d)))]
        s = [np.zeros(()), Fx.copy(), 2 * sym(outer(Fx, ux)),
             3 * sym(outer(Fx, ux, ux)) + tb * 3 * sym(outer(Fx, d))]
        if p.get("H"):
            gx = c0 * gradT[:, n]
            s[3] = s[3] + r * th[n] * (1.0 - 1.0 / p["Pr"]) * 3 * sym(outer(d, gx))
        s[2] = s[2] + sigma[n] * d
        nmax = L.feq_order
        for i in range(Q):
            feq = L.w[i] * sum(contract(a[k], Ht[i][k]) / math.factorial(k) for k in range(nmax + 1))
            S = L.w[i] * sum(contract(s[k], Ht[i][k]) / math.factorial(k) for k in range(4))
            fstar[i, n] = fl[i, n] - (fl[i, n] - feq) / tau_hat + (1.0 - 1.0 / (2.0 * tau_hat)) * S
    out = np.zeros_like(fl)
    fs = fstar.reshape((Q,) + shape)
    for i in range(Q):
        out[i] = shifted(fs[i], -L.c[i]).reshape(N)   # f(x + c) <- f*(x)
    return out


@pytest.mark.parametrize("case", ["thermal_force_H", "isothermal_SC_P"])
def test_oracle_step_equals_hermite_tensor_step(case):
    L = lattice.d2q37()
    shape = (7, 7)
    if case == "thermal_force_H":
        p = W.source_params(force=True, H=True, Pr=0.71)
        rng = np.random.default_rng(11)
        g = 1e-3 * (2 * rng.random((2,) + shape) - 1)
        fld = W.random_small("D2Q37", nx=7, ny=7, seed=4)
    else:
        p = W.source_params(force=True, g=(1e-4, -2e-4, 0.0), SC=True, P=True, isothermal=True, eos="vdw",
                            eos_a=W.VDW_A, eos_b=W.VDW_B, eos_T=0.85 * W.VDW_TC, k=0.7)
        g = None
        fld = W.random_small("D2Q37", nx=7, ny=7, seed=5, amp_rho=0.0)
        fld["rho"] = 1.1 + 5.0 * (np.arange(49).reshape(7, 7) % 3 == 0)   # gas/liquid-like contrast
    o = Oracle("D2Q37", 7, 7, 1, 0.73, p)
    o.init(fld["rho"], fld["u"], fld["theta"])
    # add a non-equilibrium part so the test is not limited to equilibrium states
    rng = np.random.default_rng(2)
    o.f += 1e-3 * L.w[:, None] * (2 * rng.random(o.f.shape) - 1)
    if g is not None:
        o.set_force_field(g)
    f = o.f.copy()
    for _ in range(3):
        f = brute_step(L, p, 0.73, f, g, shape)
        o.run(1)
        scale = np.abs(f).max()
        assert np.abs(o.f - f).max() < 1e-13 * scale, np.abs(o.f - f).max()
