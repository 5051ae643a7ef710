"""Pins of the oracle's equilibrium and source polynomials (Table 2).

P3: the projections sum_i f^eq_i He_a(xi_x) He_b(xi_y) (...) of the literal
    Table 2 equilibrium equal the Hermite coefficients of the Maxwellian,
    rho E[He_a(X)] E[He_b(Y)] with X ~ N(u_x / c0, theta), computed by a
    library Gauss-Hermite rule.  This is Eq. 2.6 including the sign of the
    theta-bar^2 term of a^(4,eq) (the sign printed in Eq. 2.6 is a typo;
    Eq. 2.2 has +1/8 theta-bar^2).  Conservation (Eq. 2.3) follows.
P4: the discrete moments of each source equal its Hermite coefficients:
    F_i (Eqs. 3.2-3.3) s1 = F, s2 = [Fu], s3 = [Fuu] + theta-bar [F delta];
    H_i (Eqs. 3.6-3.7) only s3 = rho theta (1 - 1/Pr) [delta grad theta];
    P_i (Eq. 3.12) only a trace-only s2.
    The F_i check fixes Table 2's last F term as -(c.u)(u.F)/c0^4 and the
    H_i check fixes its factor as (1 - 1/Pr).
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss, hermeval

from oracle import lattice
from oracle import solver as S
import workloads as W


def _he(n, x):
    return hermeval(x, [0] * n + [1])


def _proj(L, f, A):
    xi = L.c / L.c0
    return (f * np.prod([_he(A[a], xi[:, a]) for a in range(L.D)], axis=0)).sum()


def _maxwell_coef(rho, u_xi, theta, A):
    z, wz = hermegauss(40)
    wz = wz / wz.sum()
    return rho * np.prod([(wz * _he(A[a], u_xi[a] + np.sqrt(theta) * z)).sum() for a in range(len(A))])


@pytest.mark.parametrize("name", ["D2Q37", "D3Q39"])
def test_equilibrium_is_maxwellian_projection(name):
    L = lattice.get(name)
    rng = np.random.default_rng(7)
    for _ in range(6):
        rho = 0.5 + rng.random()
        u = 0.15 * (2 * rng.random(L.D) - 1)
        theta = 0.8 + 0.4 * rng.random()
        f = S.feq(L, rho, u, theta)
        for A in itertools.product(range(L.feq_order + 1), repeat=L.D):
            if sum(A) > L.feq_order:
                continue
            got = _proj(L, f, A)
            ref = _maxwell_coef(rho, u / L.c0, theta, A)
            assert abs(got - ref) < 1e-13 * max(1.0, abs(ref)), (A, got, ref)
        # Eq. 2.3: mass, momentum and the trace of the second moment
        cc = (L.c ** 2).sum(axis=1)
        assert abs(f.sum() - rho) < 1e-14
        assert np.allclose(L.c.T @ f, rho * u, rtol=0, atol=1e-14)
        assert abs(cc @ f - rho * ((u * u).sum() + L.D * L.cs2 * theta)) < 1e-13


def test_equilibrium_a4_sign_matters():
    """With the printed minus sign on theta-bar^2 delta^2 the xxxx coefficient
    would be rho (u^4 + 6 tb u^2 - 3 tb^2); the lattice equilibrium has + 3 tb^2."""
    L = lattice.d2q37()
    rho, u, theta = 1.0, np.array([0.0, 0.0]), 1.2
    f = S.feq(L, rho, u, theta)
    tb = theta - 1.0
    assert abs(_proj(L, f, (4, 0)) - 3 * rho * tb * tb) < 1e-13
    assert abs(_proj(L, f, (4, 0)) + 3 * rho * tb * tb) > 1e-2


def _component(T, A):
    idx = sum(([a] * A[a] for a in range(len(A))), [])
    return T[tuple(idx)] if idx else float(T)


def _delta_sym(v, D):
    """[delta v] for a vector v: delta_ab v_c + delta_ac v_b + delta_bc v_a."""
    d = np.eye(D)
    return (np.einsum("ab,c->abc", d, v) + np.einsum("ac,b->abc", d, v) + np.einsum("bc,a->abc", d, v))


@pytest.mark.parametrize("name", ["D2Q37", "D3Q39"])
def test_body_force_source_moments(name):
    L = lattice.get(name)
    D = L.D
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 0.7 + rng.random()
        u = 0.1 * (2 * rng.random(D) - 1)
        theta = 0.9 + 0.2 * rng.random()
        F = 1e-2 * (2 * rng.random(D) - 1)
        p = W.source_params(force=True)
        SF, _, _ = S.sources(L, p, 0.8, rho, u, theta, F)
        # lattice-unit moments
        assert abs(SF.sum()) < 1e-16
        assert np.allclose(L.c.T @ SF, F, rtol=0, atol=1e-16)
        M2 = np.einsum("i,ia,ib->ab", SF, L.c, L.c)
        assert np.allclose(M2, np.outer(F, u) + np.outer(u, F), rtol=0, atol=1e-16)
        # third Hermite coefficient in xi units: F_xi = F / c0, u_xi = u / c0
        Fx, ux, tb = F / L.c0, u / L.c0, theta - 1.0
        s3 = (np.einsum("a,b,c->abc", Fx, ux, ux) + np.einsum("a,b,c->abc", ux, Fx, ux)
              + np.einsum("a,b,c->abc", ux, ux, Fx) + tb * _delta_sym(Fx, D))
        for A in itertools.product(range(4), repeat=D):
            if sum(A) == 3:
                assert abs(_proj(L, SF, A) - _component(s3, A)) < 1e-15, A
            if sum(A) == 4:
                assert abs(_proj(L, SF, A)) < 1e-15, A


def test_body_force_printed_last_term_is_a_typo():
    """Table 2 prints -(c.u)(c.F)/c0^4 as the last F_i term; with it the second
    moment would lose the [Fu] coefficient of Eq. 3.2 (it cancels the second term)."""
    L = lattice.d2q37()
    rho, u, theta, F = 1.0, np.array([0.05, -0.02]), 1.0, np.array([1e-3, 2e-3])
    SF, _, _ = S.sources(L, W.source_params(force=True), 0.8, rho, u, theta, F)
    cu, cF = L.c @ u, L.c @ F
    printed = SF + L.w * (cu * (u @ F)) / L.cs2 ** 2 - L.w * cu * cF / L.cs2 ** 2
    M2 = np.einsum("i,ia,ib->ab", printed, L.c, L.c)
    assert not np.allclose(M2, np.outer(F, u) + np.outer(u, F), rtol=0, atol=1e-8)


@pytest.mark.parametrize("name", ["D2Q37", "D3Q39"])
def test_thermal_diffusion_source_moments(name):
    L = lattice.get(name)
    D = L.D
    rng = np.random.default_rng(5)
    Pr = 0.71
    for _ in range(4):
        rho, theta = 0.8 + 0.4 * rng.random(), 0.9 + 0.2 * rng.random()
        gT = 1e-2 * (2 * rng.random(D) - 1)
        p = W.source_params(H=True, Pr=Pr)
        _, SH, _ = S.sources(L, p, 0.8, rho, np.zeros(D), theta, np.zeros(D), gradT=gT)
        # only s^(3) is non-zero: s3 = rho theta (1 - 1/Pr) [delta grad_xi theta],
        # with grad_xi = c0 grad (xi-space lengths are x / c0)
        s3 = rho * theta * (1.0 - 1.0 / Pr) * _delta_sym(L.c0 * gT, D)
        for A in itertools.product(range(5), repeat=D):
            n = sum(A)
            if n > 4:
                continue
            want = _component(s3, A) if n == 3 else 0.0
            assert abs(_proj(L, SH, A) - want) < 1e-15, (A, _proj(L, SH, A), want)


@pytest.mark.parametrize("name", ["D2Q37", "D3Q39"])
def test_pressure_tensor_source_moments(name):
    L = lattice.get(name)
    D = L.D
    tau_hat, k, psi = 0.8, 0.7, 1.3
    Fsc = np.array([3e-3, -2e-3, 1e-3])[:D]
    p = W.source_params(SC=True, P=True, isothermal=True, k=k)
    _, _, SP = S.sources(L, p, tau_hat, 1.0, np.zeros(D), 1.0, np.zeros(D), Fsc=Fsc, psi=psi)
    # trace-only second coefficient sigma delta with tau = tau^ - 1/2 (Eq. 3.12 scaled by Table 2)
    sigma = -k * L.cs2 * (Fsc @ Fsc) / (D * (tau_hat - 0.5) * (-1.0) * psi * psi)
    qdeg = 9 if D == 2 else 7
    for A in itertools.product(range(4), repeat=D):
        n = sum(A)
        if n + 2 > qdeg:     # projection exact only within the quadrature degree
            continue
        want = sigma if (n == 2 and max(A) == 2) else 0.0
        assert abs(_proj(L, SP, A) - want) < 1e-16, (A, _proj(L, SP, A), want)
    # its |c|^2 moment (enters G2 of Eq. 4.5): -k c0^4 |F|^2 / (tau psi^2 G)
    cc = (L.c ** 2).sum(axis=1)
    assert abs(cc @ SP - (-k * L.cs2 ** 2 * (Fsc @ Fsc) / ((tau_hat - 0.5) * psi * psi * -1.0))) < 1e-16
