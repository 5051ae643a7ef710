"""Equations of state and the Maxwell equal-area construction (Sec. 5.4).

TEST INFRASTRUCTURE (see oracle/__init__.py).

p_EOS in lattice units, R = 1:
  van der Waals:        p = rho T / (1 - b rho) - a rho^2
  Carnahan-Starling:    p = rho T (1 + e + e^2 - e^3) / (1 - e)^3 - a rho^2,  e = b rho / 4   (Eq. 5.9)

Coexistence (Maxwell's rule, used for rho_l,0 and rho_g,0 in Eqs. 5.10-5.11):
  p(rho_g) = p(rho_l) = p*   and   int_{rho_g}^{rho_l} (p(rho) - p*) / rho^2 drho = 0
(the equal-area rule in the p-v plane with v = 1/rho).
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq, minimize_scalar


def pressure(kind: str, rho, a: float, b: float, T: float):
    rho = np.asarray(rho, dtype=np.float64)
    if kind == "vdw":
        return rho * T / (1.0 - b * rho) - a * rho * rho
    if kind == "cs":
        e = b * rho / 4.0
        return rho * T * (1.0 + e + e * e - e ** 3) / (1.0 - e) ** 3 - a * rho * rho
    raise ValueError(kind)


def _rho_max(kind: str, b: float) -> float:
    # pole of the repulsive term: b rho = 1 (vdW) or b rho / 4 = 1 (C-S)
    return (1.0 / b) if kind == "vdw" else (4.0 / b)


def _dpdrho(kind, rho, a, b, T, h=1e-7):
    return (pressure(kind, rho + h, a, b, T) - pressure(kind, rho - h, a, b, T)) / (2 * h)


def critical_temperature(kind: str, a: float, b: float) -> float:
    """T_c: the largest T at which dp/drho still touches zero."""
    rmax = _rho_max(kind, b)

    def min_slope(T):
        r = minimize_scalar(lambda x: _dpdrho(kind, x, a, b, T), bounds=(1e-6 * rmax, 0.99 * rmax),
                            method="bounded", options={"xatol": 1e-12})
        return r.fun

    lo, hi = 1e-6, 10.0
    while min_slope(hi) < 0:
        hi *= 2
    return brentq(min_slope, lo, hi, xtol=1e-14)


def spinodals(kind, a, b, T):
    """Densities of the local max and local min of p(rho) below T_c."""
    rmax = _rho_max(kind, b)
    xs = np.linspace(1e-6 * rmax, 0.999 * rmax, 200001)
    s = _dpdrho(kind, xs, a, b, T)
    idx = np.where(np.diff(np.sign(s)) != 0)[0]
    if len(idx) < 2:
        raise ValueError("no van der Waals loop at this temperature")
    r1 = brentq(lambda x: _dpdrho(kind, x, a, b, T), xs[idx[0]], xs[idx[0] + 1], xtol=1e-15)
    r2 = brentq(lambda x: _dpdrho(kind, x, a, b, T), xs[idx[1]], xs[idx[1] + 1], xtol=1e-15)
    return r1, r2


def maxwell(kind: str, a: float, b: float, T: float):
    """Coexistence densities (rho_g, rho_l) and pressure p* by the equal-area rule."""
    rmax = _rho_max(kind, b)
    s1, s2 = spinodals(kind, a, b, T)
    pmax = float(pressure(kind, s1, a, b, T))    # local max (gas spinodal)
    pmin = float(pressure(kind, s2, a, b, T))    # local min (liquid spinodal)

    def roots(ps):
        rg = brentq(lambda x: pressure(kind, x, a, b, T) - ps, 0.0, s1, xtol=1e-16)
        rl = brentq(lambda x: pressure(kind, x, a, b, T) - ps, s2, 0.9999999 * rmax, xtol=1e-15)
        return rg, rl

    def area(ps):
        rg, rl = roots(ps)
        val, _ = quad(lambda x: (pressure(kind, x, a, b, T) - ps) / (x * x), rg, rl,
                      epsabs=1e-14, epsrel=1e-13, limit=400)
        return val

    # p* lies between the spinodal pressures and above zero (the gas branch
    # starts at p(0) = 0).
    lo = max(pmin, 0.0) + 1e-12 * abs(pmax)
    hi = pmax - 1e-12 * abs(pmax)
    ps = brentq(area, lo, hi, xtol=1e-15, rtol=1e-15)
    rg, rl = roots(ps)
    return rg, rl, ps
