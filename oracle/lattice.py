"""Discrete velocity sets and Gauss-Hermite quadrature weights (oracle side).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import anything under ``oracle/``.

D2Q37 (Sec. 4.1, Table 1, Fig. 1): 37 integer velocities on the shells
|c|^2 in {0,1,2,4,5,8,9,10}.  The weights and the lattice constant c0 are the
solution of the moment conditions of a degree-9 Gauss-Hermite quadrature:
for every even a, b with a + b <= 8,

    sum_i w_i c_ix^a c_iy^b = c0^(a+b) (a-1)!! (b-1)!!,

i.e. the discrete moments of w_i with xi_i = c_i / c0 equal those of the
standard Gaussian (Eq. 2.5 needs the Hermite polynomials to stay orthogonal
on the lattice).  Odd moments vanish by the symmetry of the shells, so there
are 9 equations for 8 shell weights plus c0.  The paper writes
"c_i = xi_i / c0" in Sec. 4.1; the scaled forms of Table 2 only follow from
xi_i = c_i / c0 (integer c_i), which is the reading used here.

D3Q39 is not in the paper.  It is the standard degree-7 three-dimensional
multi-speed lattice (shells (0,0,0), (1,0,0), (1,1,1), (2,0,0), (2,2,0),
(3,0,0)); its 6 weights and c0 solve the 7 even moment conditions to order 6.

The index order inside a shell has no physical meaning; the one below follows
the grouping of Table 1.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
from scipy.optimize import fsolve


def _rot4(a: int, b: int):
    """The four 90-degree rotations of (a, b)."""
    return [(a, b), (-b, a), (-a, -b), (b, -a)]


def d2q37_velocities() -> np.ndarray:
    """Velocities of D2Q37 in the grouping of Table 1 (Sec. 4.1)."""
    v = [(0, 0)]
    for base in [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (1, 2), (3, 0), (3, 1), (1, 3)]:
        v += _rot4(*base)
    c = np.array(v, dtype=np.int64)
    assert c.shape == (37, 2) and len({tuple(x) for x in v}) == 37
    return c


def d3q39_velocities() -> np.ndarray:
    """Velocities of D3Q39: all sign/permutation images of the six shell representatives."""
    reps = [(0, 0, 0), (1, 0, 0), (1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 0, 0)]
    out = []
    for r in reps:
        imgs = set()
        for p in itertools.permutations(r):
            for s in itertools.product((1, -1), repeat=3):
                imgs.add(tuple(int(p[k] * s[k]) for k in range(3)))
        out += sorted(imgs, reverse=True)
    c = np.array(out, dtype=np.int64)
    assert c.shape == (39, 3)
    return c


def _dfact(n: int) -> int:
    """(n-1)!! for even n (the n-th moment of the standard normal); 1 for n == 0."""
    r = 1
    for k in range(n - 1, 0, -2):
        r *= k
    return r


def _shell_ids(c: np.ndarray) -> np.ndarray:
    """Shell index of each velocity: shells are the distinct |c|^2 values in
    order of appearance (D2Q37 and D3Q39 have one orbit per |c|^2)."""
    n2 = (c * c).sum(axis=1)
    order = []
    for v in n2:
        if v not in order:
            order.append(int(v))
    return np.array([order.index(int(v)) for v in n2])


def _moment_conditions(D: int, max_order: int):
    """Exponent tuples (sorted descending, even entries) for the isotropic moment equations."""
    conds = []
    for order in range(0, max_order + 1, 2):
        for parts in itertools.combinations_with_replacement(range(order, -1, -2), D):
            if sum(parts) == order and list(parts) == sorted(parts, reverse=True):
                conds.append(tuple(parts))
    return conds


def solve_weights(c: np.ndarray, max_order: int, guess_w, guess_cs2: float):
    """Solve the moment equations for the shell weights and c0^2.

    Unknowns: one weight per shell and s = c0^2.  Equation for exponents e:
    sum_i W_shell(i) prod_k c_ik^e_k - s^(|e|/2) prod_k (e_k-1)!! = 0.
    """
    D = c.shape[1]
    sid = _shell_ids(c)
    nsh = sid.max() + 1
    conds = _moment_conditions(D, max_order)
    assert len(conds) == nsh + 1, (len(conds), nsh)
    cf = c.astype(np.float64)
    # M[j, k] = sum over shell k of prod c^e_j
    M = np.zeros((len(conds), nsh))
    rhs_coef = np.zeros(len(conds))
    half = np.zeros(len(conds))
    for j, e in enumerate(conds):
        mono = np.prod([cf[:, k] ** e[k] for k in range(D)], axis=0)
        for k in range(nsh):
            M[j, k] = mono[sid == k].sum()
        rhs_coef[j] = np.prod([_dfact(ek) for ek in e])
        half[j] = sum(e) / 2

    def resid(x):
        W, s = x[:nsh], x[nsh]
        return M @ W - rhs_coef * s ** half

    x0 = np.concatenate([np.asarray(guess_w, float), [guess_cs2]])
    x, info, ier, msg = fsolve(resid, x0, full_output=True, xtol=1e-14)
    # fsolve may stop on its step tolerance after reaching round-off; the
    # residual is what decides.
    if np.max(np.abs(resid(x))) > 1e-13:
        raise RuntimeError(f"weight solve failed: {msg}")
    W, s = x[:nsh], x[nsh]
    return W[sid], float(s)


@dataclass(frozen=True)
class Lattice:
    name: str
    D: int
    c: np.ndarray     # (Q, D) int64
    w: np.ndarray     # (Q,) float64
    cs2: float        # c0^2

    @property
    def Q(self) -> int:
        return self.c.shape[0]

    @property
    def c0(self) -> float:
        return float(np.sqrt(self.cs2))

    @property
    def feq_order(self) -> int:
        # Eq. 2.2 to 4th order needs a degree-9 quadrature (D2Q37); the degree-7
        # D3Q39 integrates Hermite products only up to m + n <= 7, so its
        # equilibrium is truncated after the 3rd-order terms.
        return 4 if self.name == "D2Q37" else 3


_CACHE: dict = {}


def d2q37() -> Lattice:
    if "D2Q37" not in _CACHE:
        c = d2q37_velocities()
        # Deliberately coarse start (one significant digit), so that agreement
        # with every printed digit of Table 1 is a result of the solve.
        guess = [0.2, 0.1, 0.06, 0.01, 0.005, 0.001, 0.0002, 0.0003]
        w, s = solve_weights(c, 8, guess, 0.7)
        _CACHE["D2Q37"] = Lattice("D2Q37", 2, c, w, s)
    return _CACHE["D2Q37"]


def d3q39() -> Lattice:
    if "D3Q39" not in _CACHE:
        c = d3q39_velocities()
        guess = [0.1, 0.1, 0.04, 0.01, 0.002, 0.0006]
        w, s = solve_weights(c, 6, guess, 0.7)
        _CACHE["D3Q39"] = Lattice("D3Q39", 3, c, w, s)
    return _CACHE["D3Q39"]


def get(name: str) -> Lattice:
    return {"D2Q37": d2q37, "D3Q39": d3q39}[name]()
