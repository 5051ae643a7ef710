"""ctypes front end of the FP64 C oracle (oracle/hlbm_oracle.c).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import anything under ``oracle/``.

Field layout (same convention as the public API, but double precision):
  2D: rho, theta [ny, nx]; u [2, ny, nx]
  3D: rho, theta [nz, ny, nx]; u [3, nz, ny, nx]
Source parameters are a dict with the keys of ``workloads.source_params``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

from . import lattice as _lat

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "hlbm_oracle.c"
_BUILD = _HERE / "_build"
_SO = _BUILD / "libhlbm_oracle.so"


def build(force: bool = False) -> Path:
    """Compile the oracle (plain C11, FP64, OpenMP) into oracle/_build/."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(_SO), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


class _Lat(C.Structure):
    _fields_ = [("D", C.c_int), ("Q", C.c_int), ("c", (C.c_int * 3) * 64),
                ("w", C.c_double * 64), ("cs2", C.c_double)]


class _Par(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("tau_hat", C.c_double),
                ("feq_order", C.c_int), ("thermal", C.c_int), ("use_force", C.c_int),
                ("g_uniform", C.c_double * 3), ("use_H", C.c_int), ("Pr", C.c_double),
                ("use_SC", C.c_int), ("use_P", C.c_int), ("eos", C.c_int),
                ("eos_a", C.c_double), ("eos_b", C.c_double), ("eos_T", C.c_double),
                ("k", C.c_double), ("walls", C.c_int), ("wall_rule", C.c_int),
                ("wall_u", (C.c_double * 3) * 2), ("wall_theta", C.c_double * 2), ("lag", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        dp = C.POINTER(C.c_double)
        _lib.or_step.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, dp, dp]
        _lib.or_run.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, C.c_int, dp, dp]
        _lib.or_macros_psi.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.or_wall_complete.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, dp]
        _lib.or_init.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, dp]
        _lib.or_macros.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.or_feq.argtypes = [C.POINTER(_Lat), C.c_int, C.c_double, dp, C.c_double, dp]
        _lib.or_sources.argtypes = [C.POINTER(_Lat), C.POINTER(_Par), C.c_double, dp, C.c_double,
                                    dp, dp, dp, C.c_double, dp, dp, dp]
        _lib.or_peos.argtypes = [C.POINTER(_Par), C.c_double]
        _lib.or_peos.restype = C.c_double
        _lib.or_psi.argtypes = [C.POINTER(_Par), C.c_double, C.c_double]
        _lib.or_psi.restype = C.c_double
        _lib.or_set_threads.argtypes = [C.c_int]
        _lib.or_get_threads.restype = C.c_int
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_lattice_struct(L: _lat.Lattice) -> _Lat:
    s = _Lat()
    s.D, s.Q = L.D, L.Q
    for i in range(L.Q):
        for a in range(3):
            s.c[i][a] = int(L.c[i, a]) if a < L.D else 0
        s.w[i] = float(L.w[i])
    s.cs2 = float(L.cs2)
    return s


def make_params_struct(L: _lat.Lattice, nx, ny, nz, tau_hat, p: dict) -> _Par:
    s = _Par()
    s.nx, s.ny, s.nz = nx, ny, nz
    s.tau_hat = float(tau_hat)
    s.feq_order = L.feq_order
    s.thermal = 0 if p.get("isothermal", False) else 1
    s.use_force = 1 if p.get("force", False) else 0
    g = list(p.get("g", (0.0, 0.0, 0.0))) + [0.0] * 3
    for a in range(3):
        s.g_uniform[a] = float(g[a])
    s.use_H = 1 if p.get("H", False) else 0
    s.Pr = float(p.get("Pr", 1.0))
    s.use_SC = 1 if p.get("SC", False) else 0
    s.use_P = 1 if p.get("P", False) else 0
    s.eos = {"vdw": 0, "cs": 1}[p.get("eos", "vdw")]
    s.eos_a = float(p.get("eos_a", 0.0))
    s.eos_b = float(p.get("eos_b", 0.0))
    s.eos_T = float(p.get("eos_T", 0.0))
    s.k = float(p.get("k", 0.0))
    s.walls = 1 if p.get("walls", False) else 0
    s.wall_rule = int(p.get("wall_rule", 0))
    wu = p.get("wall_u", ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)))
    wt = p.get("wall_theta", (1.0, 1.0))
    for side in range(2):
        v = list(wu[side]) + [0.0] * 3
        for a in range(3):
            s.wall_u[side][a] = float(v[a])
        s.wall_theta[side] = float(wt[side])
    s.lag = 1 if p.get("lag", False) else 0
    return s


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


class Oracle:
    """Plain FP64 solver: state f[Q, N] of shifted populations after streaming."""

    def __init__(self, lattice: str, nx: int, ny: int, nz: int, tau_hat: float, params: dict):
        self.L = _lat.get(lattice)
        self.nx, self.ny, self.nz = nx, ny, max(1, nz)
        if self.L.D == 2:
            assert self.nz == 1
        self.N = self.nx * self.ny * self.nz
        self.tau_hat = tau_hat
        self.params = dict(params)
        self._ls = make_lattice_struct(self.L)
        self._ps = make_params_struct(self.L, self.nx, self.ny, self.nz, tau_hat, self.params)
        self.f = np.zeros((self.L.Q, self.N))
        self._tmp = np.zeros_like(self.f)
        self.g = None
        self.step_count = 0
        # walls: the previous step's moments [rho, u_1..u_D, theta] (targets of Eqs. 4.7-4.8)
        self.walls = bool(self.params.get("walls", False))
        self.bcm = np.zeros((self.L.D + 2, self.N)) if self.walls else None
        # single-pass variant: the previous step's theta and psi [2, N]
        self.lag = bool(self.params.get("lag", False))
        self.lagf = np.zeros((2, self.N)) if self.lag else None

    @property
    def shape(self):
        return (self.ny, self.nx) if self.L.D == 2 else (self.nz, self.ny, self.nx)

    def _flat(self, a, comps=None):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if comps is None:
            return a.reshape(self.N)
        return a.reshape(comps, self.N)

    def init(self, rho, u, theta):
        r, uu, t = self._flat(rho), self._flat(u, self.L.D), self._flat(theta)
        lib().or_init(C.byref(self._ls), C.byref(self._ps), _ptr(r), _ptr(uu), _ptr(t), _ptr(self.f))
        if self.walls:
            self.bcm[0], self.bcm[1:1 + self.L.D], self.bcm[1 + self.L.D] = r, uu, t
        if self.lag:
            self.lagf[0] = t
            self.lagf[1] = 0.0
            if self.params.get("SC"):
                from . import eos
                p = self.params
                pe = eos.pressure(p.get("eos", "vdw"), r, p["eos_a"], p["eos_b"], p["eos_T"])
                self.lagf[1] = np.sqrt(np.maximum(2.0 * (pe - r * self.L.cs2) / (-1.0 * self.L.cs2), 0.0))
        self.step_count = 0

    def set_force_field(self, g):
        """Acceleration field [D, ...] (force density F = rho g); None = uniform params['g']."""
        self.g = None if g is None else self._flat(g, self.L.D).copy()

    def run(self, nsteps: int):
        rc = lib().or_run(C.byref(self._ls), C.byref(self._ps), _ptr(self.f), _ptr(self._tmp),
                          _ptr(self.g), int(nsteps), _ptr(self.bcm), _ptr(self.lagf))
        if rc != 0:
            raise MemoryError("oracle step failed to allocate")
        self.step_count += nsteps

    def macros(self) -> dict:
        N, D = self.N, self.L.D
        out = {k: np.zeros(N) for k in ("rho", "theta", "psi")}
        for k in ("u", "F", "Fsc"):
            out[k] = np.zeros((3, N))
        f = self.f
        if self.walls:
            # the state holds what streaming delivered; the wall completes it first
            f = np.empty_like(self.f)
            lib().or_wall_complete(C.byref(self._ls), C.byref(self._ps), _ptr(self.f), _ptr(f), _ptr(self.g),
                                   _ptr(self.bcm))
        lib().or_macros_psi(C.byref(self._ls), C.byref(self._ps), _ptr(f), _ptr(self.g),
                            _ptr(self.lagf[1].copy()) if self.lag else None,
                        _ptr(out["rho"]), _ptr(out["u"]), _ptr(out["theta"]), _ptr(out["F"]),
                        _ptr(out["psi"]), _ptr(out["Fsc"]))
        res = {}
        for k, v in out.items():
            res[k] = v[:D].reshape((D,) + self.shape) if v.ndim == 2 else v.reshape(self.shape)
        return res

    def moments(self):
        m = self.macros()
        return m["rho"], m["u"], m["theta"]

    def diag(self) -> np.ndarray:
        """[mass, momentum_1..D, energy] with momentum = sum rho u and
        energy = sum (rho |u|^2 + D rho c0^2 theta) / 2 (Eq. 2.3 invariants)."""
        rho, u, th = self.moments()
        D = self.L.D
        mom = [float((rho * u[a]).sum()) for a in range(D)]
        en = float((0.5 * rho * ((u * u).sum(axis=0) + D * self.L.cs2 * th)).sum())
        return np.array([float(rho.sum())] + mom + [en])


def feq(L: _lat.Lattice, rho: float, u, theta: float, order: int | None = None) -> np.ndarray:
    """f^eq_i at one node (Table 2, first row)."""
    out = np.zeros(L.Q)
    uu = np.zeros(3)
    uu[:L.D] = u
    lib().or_feq(C.byref(make_lattice_struct(L)), L.feq_order if order is None else order,
                 float(rho), _ptr(uu), float(theta), _ptr(out))
    return out


def sources(L: _lat.Lattice, params: dict, tau_hat: float, rho, u, theta, F, gradT=None, Fsc=None, psi=0.0):
    """(F_i, H_i, P_i) at one node (Table 2, rows 2-4)."""
    ps = make_params_struct(L, 1, 1, 1, tau_hat, params)
    def v3(x):
        a = np.zeros(3)
        if x is not None:
            a[:L.D] = x
        return a
    SF, SH, SP = np.zeros(L.Q), np.zeros(L.Q), np.zeros(L.Q)
    lib().or_sources(C.byref(make_lattice_struct(L)), C.byref(ps), float(rho), _ptr(v3(u)), float(theta),
                     _ptr(v3(F)), _ptr(v3(gradT)), _ptr(v3(Fsc)), float(psi), _ptr(SF), _ptr(SH), _ptr(SP))
    return SF, SH, SP


def peos(params: dict, rho: float) -> float:
    ps = make_params_struct(_lat.d2q37(), 1, 1, 1, 1.0, params)
    return float(lib().or_peos(C.byref(ps), float(rho)))


def psi(params: dict, cs2: float, rho: float) -> float:
    ps = make_params_struct(_lat.d2q37(), 1, 1, 1, 1.0, params)
    return float(lib().or_psi(C.byref(ps), float(cs2), float(rho)))
