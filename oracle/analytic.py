"""Closed forms used as physics pins of the oracle.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Transport coefficients of the shifted scheme (Eqs. 4.3-4.4; Sec. 5.1 states
nu = c0^2 (tau^ - 1/2) for theta0 = 1): kinematic viscosity
nu = c0^2 theta0 (tau^ - 1/2); with the thermal diffusion source H_i the
thermal diffusivity is nu / Pr (Eqs. 3.4-3.6), and BGK alone gives Pr = 1.
"""
from __future__ import annotations

import numpy as np


def viscosity(cs2: float, tau_hat: float, theta0: float = 1.0) -> float:
    return cs2 * theta0 * (tau_hat - 0.5)


def kolmogorov_ux(y, t: float, g0: float, nu: float, n: int):
    """Start-up of Kolmogorov flow from rest under g_x = g0 sin(k y), k = 2 pi / n:
    u_x = g0 / (nu k^2) (1 - exp(-nu k^2 t)) sin(k y) (incompressible limit)."""
    k = 2.0 * np.pi / n
    return g0 / (nu * k * k) * (1.0 - np.exp(-nu * k * k * t)) * np.sin(k * np.asarray(y, float))


def shear_wave_rate(nu: float, n: int) -> float:
    k = 2.0 * np.pi / n
    return nu * k * k


def entropy_mode_rate(nu: float, Pr: float, n: int) -> float:
    k = 2.0 * np.pi / n
    return nu / Pr * k * k
