"""Seeded synthetic inputs for the lattice Boltzmann step.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  It holds none of the method's arithmetic: it only builds
initial macroscopic fields (rho, u, theta), body-force (acceleration) fields
and source parameter sets shaped like the paper's test cases (Sec. 5) and the
workloads this library is benchmarked on.  Random numbers come from a
counter-based SplitMix64 (Steele, Lea and Flood, 2014), so every array is a
pure function of (seed, index).

Field layout: 2D rho/theta [ny, nx], u [2, ny, nx]; 3D rho/theta
[nz, ny, nx], u [3, nz, ny, nx]; float64 arrays holding FP32-representable
values (the library's API takes FP32, so both sides see identical inputs).  A force field is an acceleration
g [D, ...] (force density F = rho g).

Source parameters (dict, keys mirror hlbm_source_params):
  force (bool), g (uniform acceleration, used when no field is given),
  H (bool), Pr, SC (bool), P (bool), isothermal (bool),
  eos ('vdw' | 'cs'), eos_a, eos_b, eos_T, k, rho0 (storage reference density).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """Counter-based SplitMix64: output i = mix(seed + (i + 1) * golden)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# Coexistence densities (rho_g, rho_l) of the van der Waals EOS a = 9/49,
# b = 2/21 (T_c = 4/7) from Maxwell's equal-area rule, per reduced
# temperature T/T_c.  Checked against the equal-area solve by the tests.
VDW_A = 9.0 / 49.0
VDW_B = 2.0 / 21.0
VDW_TC = 4.0 / 7.0
VDW_COEXIST = {
    0.70: (0.448078055830254, 7.491548919770),
    0.75: (0.620231522179000, 7.148238314517),
    0.80: (0.838834226443818, 6.764470400099),
    0.85: (1.119054875815994, 6.324991145677),
    0.90: (1.490095732034194, 5.800445741994),
    0.95: (2.026552243876127, 5.116045703149),
}

# Carnahan-Starling EOS as printed for Sec. 5.4 (Eq. 5.9): a = 0.25, b = 4;
# T_c and the coexistence densities from the oracle's Maxwell solver (checked
# against it by the tests).
CS_A = 0.25
CS_B = 4.0
CS_TC = 0.023582175788041854
CS_COEXIST = {
    0.70: (0.009294146227023828, 0.3581309411215158),
    0.75: (0.014526084623691983, 0.3332415984642653),
    0.80: (0.021723243437775562, 0.3071956822831783),
    0.85: (0.03158177953528134, 0.2792620941620207),
    0.90: (0.04542119811463903, 0.24808424109070054),
    0.95: (0.06661162931376641, 0.21025422466496013),
}

# D3Q39 lattice constant squared (the degree-7 lattice has c0^2 = 2/3); only
# used here to express the Taylor-Green pressure field and Mach number in
# lattice units.
_CS2_D3Q39 = 2.0 / 3.0
# D2Q37 lattice constant squared (Table 1: c0 = 0.83544 to the printed digits;
# the solved quadrature's value, checked against the oracle's lattice by the
# tests); only used to turn the viscosities the paper quotes for its wall
# cases (Sec. 5.1-5.3, nu = c0^2 (tau^ - 1/2)) into tau^.
CS2_D2Q37 = 0.6979533220196835


def source_params(**kw) -> dict:
    p = dict(force=False, g=(0.0, 0.0, 0.0), H=False, Pr=1.0, SC=False, P=False,
             isothermal=False, eos="vdw", eos_a=0.0, eos_b=0.0, eos_T=0.0, k=0.0, rho0=1.0)
    p.update(kw)
    return p


def fp32(a):
    """Round to the nearest FP32 value (kept as float64): the library takes FP32
    fields, so both sides start from exactly the same numbers."""
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


@dataclass
class Case:
    name: str
    lattice: str
    nx: int
    ny: int
    nz: int
    tau_hat: float
    params: dict
    rho: np.ndarray
    u: np.ndarray
    theta: np.ndarray
    gfield: np.ndarray | None = None
    steps: int = 100
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.rho, self.u, self.theta = fp32(self.rho), fp32(self.u), fp32(self.theta)
        self.gfield = fp32(self.gfield)

    @property
    def D(self) -> int:
        return 2 if self.lattice == "D2Q37" else 3

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


def kolmogorov(n: int = 64, tau_hat: float = 0.8, g0: float = 1e-5, steps: int = 2000,
               nx: int | None = None, ny: int | None = None) -> Case:
    """Kolmogorov flow from rest: g_x(y) = g0 sin(2 pi y / ny), theta0 = rho0 = 1, periodic."""
    nx = nx or n
    ny = ny or n
    y = np.arange(ny, dtype=np.float64)
    g = np.zeros((2, ny, nx))
    g[0] = (g0 * np.sin(2.0 * np.pi * y / ny))[:, None]
    return Case("kolmogorov", "D2Q37", nx, ny, 1, tau_hat,
                source_params(force=True, rho0=1.0),
                np.ones((ny, nx)), np.zeros((2, ny, nx)), np.ones((ny, nx)), g, steps,
                meta=dict(g0=g0))


def thermal_decay(n: int = 1024, tau_hat: float = 0.7, Pr: float = 0.71, seed: int = 0,
                  eps_T: float = 0.01, u0: float = 0.01, noise: float = 1e-6,
                  nx: int | None = None, ny: int | None = None, H: bool = True) -> Case:
    """theta = 1 + eps_T sin(2 pi x / nx), rho = 1 / theta (isobaric), u_x = u0 sin(2 pi y / ny),
    plus seeded noise of amplitude `noise` on rho (uniform in [-noise, noise))."""
    nx = nx or n
    ny = ny or n
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    theta = np.broadcast_to(1.0 + eps_T * np.sin(2.0 * np.pi * x / nx), (ny, nx)).copy()
    rho = 1.0 / theta
    if noise:
        rho = rho + noise * (2.0 * uniform01(seed, nx * ny).reshape(ny, nx) - 1.0)
    u = np.zeros((2, ny, nx))
    u[0] = (u0 * np.sin(2.0 * np.pi * y / ny))[:, None]
    return Case("thermal", "D2Q37", nx, ny, 1, tau_hat,
                source_params(H=H, Pr=Pr, rho0=1.0), rho, u, theta, None, 100,
                meta=dict(seed=seed, eps_T=eps_T, u0=u0))


def _multiphase_params(Tr: float, k: float, rho_g: float, rho_l: float, eos: str = "vdw") -> dict:
    # Stored populations are deviations from rho0.  u = j / rho divides their
    # absolute rounding error by the density, so the gas (the smaller density)
    # is the reference: its populations are stored as the smallest numbers.
    a, b, tc = (VDW_A, VDW_B, VDW_TC) if eos == "vdw" else (CS_A, CS_B, CS_TC)
    return source_params(SC=True, P=True, isothermal=True, eos=eos, eos_a=a, eos_b=b,
                         eos_T=Tr * tc, k=k, rho0=rho_g)


def _coexistence(eos: str, Tr: float):
    return (VDW_COEXIST if eos == "vdw" else CS_COEXIST)[round(Tr, 2)]


def droplet(n: int = 512, tau_hat: float = 0.8, Tr: float = 0.85, k: float = 0.01,
            r0: float | None = None, W: float = 5.0, steps: int = 20000,
            nx: int | None = None, ny: int | None = None, eos: str = "vdw") -> Case:
    """Liquid disk (Eq. 5.11, droplet branch) of radius r0 centred at (nx/2, ny/2),
    tanh interface of width W, coexistence densities from Maxwell's rule;
    van der Waals (eos="vdw") or Carnahan-Starling (eos="cs", Eq. 5.9)."""
    nx = nx or n
    ny = ny or n
    r0 = 100.0 if r0 is None else r0
    rho_g, rho_l = _coexistence(eos, Tr)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    d = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2)
    rho = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (d - r0) / W)
    return Case("droplet", "D2Q37", nx, ny, 1, tau_hat, _multiphase_params(Tr, k, rho_g, rho_l, eos),
                rho, np.zeros((2, ny, nx)), np.ones((ny, nx)), None, steps,
                meta=dict(Tr=Tr, rho_g=rho_g, rho_l=rho_l, r0=r0, W=W, eos=eos))


def flat_interface(nx: int = 8, ny: int = 200, tau_hat: float = 0.8, Tr: float = 0.85,
                   k: float = 0.01, W: float = 5.0, eos: str = "vdw") -> Case:
    """Liquid slab between y = ny/4 and 3 ny/4 (Eq. 5.10 with the 50 x 200 geometry of Sec. 5.4)."""
    rho_g, rho_l = _coexistence(eos, Tr)
    y = np.arange(ny, dtype=np.float64)
    prof = rho_g + 0.5 * (rho_l - rho_g) * np.abs(np.tanh(2.0 * (y - ny / 4.0) / W)
                                                  - np.tanh(2.0 * (y - 3.0 * ny / 4.0) / W))
    rho = np.broadcast_to(prof[:, None], (ny, nx)).copy()
    return Case("flat_interface", "D2Q37", nx, ny, 1, tau_hat, _multiphase_params(Tr, k, rho_g, rho_l, eos),
                rho, np.zeros((2, ny, nx)), np.ones((ny, nx)), None, 5000,
                meta=dict(Tr=Tr, rho_g=rho_g, rho_l=rho_l, eos=eos))


def shear_wave(nx: int = 8, ny: int = 128, tau_hat: float = 0.8, u0: float = 1e-3) -> Case:
    """u_x = u0 sin(2 pi y / ny), rho = theta = 1."""
    y = np.arange(ny, dtype=np.float64)
    u = np.zeros((2, ny, nx))
    u[0] = (u0 * np.sin(2.0 * np.pi * y / ny))[:, None]
    return Case("shear_wave", "D2Q37", nx, ny, 1, tau_hat, source_params(rho0=1.0),
                np.ones((ny, nx)), u, np.ones((ny, nx)), None, 1000, meta=dict(u0=u0))


def random_small(lattice: str = "D2Q37", nx: int = 13, ny: int = 11, nz: int = 1, seed: int = 1,
                 amp_rho: float = 0.05, amp_u: float = 0.05, amp_T: float = 0.05) -> dict:
    """Smooth-free random fields for unit-level checks (not a physical case)."""
    D = 2 if lattice == "D2Q37" else 3
    shape = (ny, nx) if D == 2 else (nz, ny, nx)
    N = int(np.prod(shape))
    r = uniform01(seed, (D + 2) * N).reshape(D + 2, *shape)
    rho = 1.0 + amp_rho * (2 * r[0] - 1)
    u = amp_u * (2 * r[1:1 + D] - 1)
    theta = 1.0 + amp_T * (2 * r[D + 1] - 1)
    return dict(rho=rho, u=u, theta=theta)


def taylor_green_3d(n: int = 128, tau_hat: float = 0.6, Ma: float = 0.3, steps: int = 400) -> Case:
    """Compressible Taylor-Green vortex on D3Q39.

    U = Ma c0 sqrt(gamma theta0), gamma = (D + 2) / D = 5/3 (adiabatic sound
    speed of the thermal model); u = U (sin x cos y cos z, -cos x sin y cos z, 0)
    with x = 2 pi i / n; theta = 1 and rho = p / c0^2 with
    p = c0^2 + (U^2 / 16)(cos 2x + cos 2y)(cos 2z + 2)."""
    cs2 = _CS2_D3Q39
    U = Ma * math.sqrt(cs2 * 5.0 / 3.0)
    s = 2.0 * np.pi * np.arange(n) / n
    z, y, x = np.meshgrid(s, s, s, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = U * np.sin(x) * np.cos(y) * np.cos(z)
    u[1] = -U * np.cos(x) * np.sin(y) * np.cos(z)
    p = cs2 + (U * U / 16.0) * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = p / cs2
    return Case("taylor_green", "D3Q39", n, n, n, tau_hat, source_params(force=True, rho0=1.0),
                rho, u, np.ones((n, n, n)), np.zeros((3, n, n, n)), steps, meta=dict(U=U, Ma=Ma))


def batched(n_domains: int = 256, seed: int = 0, nmin: int = 32, nmax: int = 256) -> list[Case]:
    """Independent periodic D2Q37 domains of uneven sizes and parameters.

    Domain i: Kolmogorov flow with H_i (even i) or a vdW droplet (odd i);
    side N ~ U{nmin..nmax}; tau^ ~ U[0.55, 1.2] (droplets: at least 0.7);
    g ~ log-U[1e-6, 1e-4]; Pr ~ U[0.71, 1.41]; T/T_c drawn from the tabulated
    reduced temperatures 0.80..0.95 (with k = 0.01 and width 5, droplets at
    T/T_c <= 0.75 and tau^ = 0.7 reach |u| > 0.3 and blow up in the FP64
    oracle itself); droplet radius 0.2 N, width 5."""
    r = uniform01(seed, 6 * n_domains).reshape(n_domains, 6)
    trs = [t for t in sorted(VDW_COEXIST) if t >= 0.80]
    cases = []
    for i in range(n_domains):
        N = nmin + int(r[i, 0] * (nmax - nmin + 1))
        tau = 0.55 + 0.65 * r[i, 1]
        if i % 2 == 0:
            g0 = 10.0 ** (-6.0 + 2.0 * r[i, 2])
            Pr = 0.71 + 0.70 * r[i, 3]
            c = kolmogorov(N, tau, g0, steps=1000)
            c.params.update(H=True, Pr=Pr)
            c.name = f"kolmogorov{i}"
        else:
            Tr = trs[min(len(trs) - 1, int(r[i, 4] * len(trs)))]
            c = droplet(N, max(tau, 0.7), Tr, k=0.01, r0=0.2 * N, W=5.0, steps=1000)
            c.name = f"droplet{i}"
        cases.append(c)
    return cases


def _wall_params(u_bottom=(0.0, 0.0), u_top=(0.0, 0.0), theta_bottom=1.0, theta_top=1.0, **kw) -> dict:
    return source_params(walls=True, wall_u=(tuple(u_bottom) + (0.0,), tuple(u_top) + (0.0,)),
                         wall_theta=(theta_bottom, theta_top), **kw)


def couette(nx: int = 50, ny: int = 56, nu: float = 0.01, Re: float = 100.0, Pr: float = 0.71,
            Ec: float = 10.0, theta_top: float = 0.8, steps: int = 1000, developed: bool = False) -> Case:
    """Thermal Couette flow (Sec. 5.1, Fig. 3): walls below row 0 and above row
    ny - 1 with the solid-liquid interfaces half a cell inside the wall rows,
    H = ny - 2 (50 x 56 gives the paper's 54); the top wall moves at
    u0 = Re nu / H and holds theta_top, the bottom wall is at rest at
    theta_top - Delta theta with Ec = u0^2 / (c_p Delta theta), c_p = 2 c0^2
    (Eq. 5.3, the specific heat at constant pressure of the D2Q37 gas in units
    of theta).  nu = c0^2 (tau^ - 1/2) as in Sec. 5.1.  The fluid starts at
    rest at theta_top (Sec. 5.1) with rho = 1, or (developed=True) in the
    profiles of Eqs. 5.1-5.2 (y* from the bottom interface) with
    rho theta = theta_top.  The thermal source H_i sets Pr."""
    H = ny - 2
    u0 = Re * nu / H
    dth = u0 * u0 / (2.0 * CS2_D2Q37 * Ec)
    tau = 0.5 + nu / CS2_D2Q37
    p = _wall_params(u_top=(u0, 0.0), theta_bottom=theta_top - dth, theta_top=theta_top,
                     H=(Pr != 1.0), Pr=Pr, rho0=1.0)
    rho, u, theta = np.ones((ny, nx)), np.zeros((2, ny, nx)), np.full((ny, nx), theta_top)
    if developed:
        ys = ((np.arange(ny, dtype=np.float64) - 0.5) / H)[:, None]
        u[0] = np.broadcast_to(u0 * ys, (ny, nx))
        theta = np.broadcast_to(theta_top - dth + dth * (ys + 0.5 * Pr * Ec * ys * (1.0 - ys)), (ny, nx)).copy()
        rho = theta_top / theta
    return Case("couette", "D2Q37", nx, ny, 1, tau, p, rho, u, theta, None, steps,
                meta=dict(H=H, u0=u0, dtheta=dth, Ec=Ec, Pr=Pr, nu=nu, theta_bottom=theta_top - dth,
                          theta_top=theta_top))


def poiseuille(nx: int = 50, ny: int = 56, nu: float = 0.01, Re: float = 100.0, Pr: float = 0.71,
               Ec: float = 10.0, theta_top: float = 0.8, steps: int = 1000, developed: bool = False) -> Case:
    """Thermal Poiseuille flow (Sec. 5.2, Fig. 6): both walls at rest, the top at
    theta_top, the bottom Delta theta colder; a uniform acceleration g along x
    drives the flow.  Centre-line speed u_c = Re nu / H, g = 8 nu u_c / H^2
    (Eq. 5.4 with rho0 theta0 = 1), Ec = u_c^2 / (c_p Delta theta).  Geometry,
    nu and the initial state as in couette() (developed: Eqs. 5.4-5.5)."""
    H = ny - 2
    uc = Re * nu / H
    g = 8.0 * nu * uc / (H * H)
    dth = uc * uc / (2.0 * CS2_D2Q37 * Ec)
    tau = 0.5 + nu / CS2_D2Q37
    p = _wall_params(theta_bottom=theta_top - dth, theta_top=theta_top, force=True, g=(g, 0.0, 0.0),
                     H=(Pr != 1.0), Pr=Pr, rho0=1.0)
    rho, u, theta = np.ones((ny, nx)), np.zeros((2, ny, nx)), np.full((ny, nx), theta_top)
    if developed:
        ys = ((np.arange(ny, dtype=np.float64) - 0.5) / H)[:, None]
        u[0] = np.broadcast_to(4.0 * uc * ys * (1.0 - ys), (ny, nx))
        theta = np.broadcast_to(theta_top - dth + dth * (ys + Pr * Ec / 3.0 * (1.0 - (1.0 - 2.0 * ys) ** 4)),
                                (ny, nx)).copy()
        rho = theta_top / theta
    return Case("poiseuille", "D2Q37", nx, ny, 1, tau, p, rho, u, theta, None, steps,
                meta=dict(H=H, uc=uc, g=g, dtheta=dth, Ec=Ec, Pr=Pr, nu=nu))


def rayleigh_benard(nx: int = 200, ny: int = 102, Ra: float = 10000.0, Pr: float = 1.41, nu: float = 0.04,
                    theta_hot: float = 1.4, theta_cold: float = 1.0, steps: int = 1000,
                    roll: float = 0.0) -> Case:
    """Rayleigh-Benard convection (Sec. 5.3, Fig. 9): L = nx, H = ny - 2 (200 x 102
    gives the paper's L = 200, H = 100), periodic in x, the bottom wall hot and
    the top wall cold, gravity -g along y with g from Eq. 5.6,
    Ra = 2 Pr g (theta_h - theta_c) H^3 / (nu^2 (theta_h + theta_c)).
    Eq. 5.6 takes the expansion coefficient at the mean temperature
    theta_m = (theta_h + theta_c) / 2, so nu is read at theta_m too: the
    model's viscosity c0^2 theta (tau^ - 1/2) equals nu at theta_m.
    Initial temperature (Eq. 5.7, y measured up from the bottom interface, hot
    at the bottom): theta = theta_h - (theta_h - theta_c) y / H
    + 0.01 (theta_h - theta_c) sin(pi x / L) sin(pi y / H); rho = 1 / theta
    (uniform pressure), u = 0, or (roll > 0) the pair of convection rolls of
    stream function roll (H / pi) sin(2 pi x / L) sin(pi y / H) (peak speed
    about roll).  Body force F_i and H_i are on (Sec. 5.3)."""
    H = ny - 2
    dth = theta_hot - theta_cold
    g = Ra * nu * nu * (theta_hot + theta_cold) / (2.0 * Pr * dth * H ** 3)
    tau = 0.5 + nu / (CS2_D2Q37 * 0.5 * (theta_hot + theta_cold))
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None] - 0.5          # distance from the bottom interface
    theta = theta_hot - dth * y / H + 0.01 * dth * np.sin(np.pi * x / nx) * np.sin(np.pi * y / H)
    theta = np.broadcast_to(theta, (ny, nx)).copy()
    p = _wall_params(theta_bottom=theta_hot, theta_top=theta_cold, force=True, g=(0.0, -g, 0.0),
                     H=(Pr != 1.0), Pr=Pr, rho0=1.0 / theta_cold)
    u = np.zeros((2, ny, nx))
    if roll:
        kx, ky = 2.0 * np.pi / nx, np.pi / H
        u[0] = np.broadcast_to(roll * (ky * H / np.pi) * np.sin(kx * x) * np.cos(ky * y), (ny, nx))
        u[1] = np.broadcast_to(-roll * (kx * H / np.pi) * np.cos(kx * x) * np.sin(ky * y), (ny, nx))
    return Case("rayleigh_benard", "D2Q37", nx, ny, 1, tau, p, 1.0 / theta, u, theta,
                None, steps, meta=dict(H=H, L=nx, Ra=Ra, g=g, dtheta=dth, Pr=Pr, nu=nu))
