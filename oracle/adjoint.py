"""FP64 discrete adjoint of the body-force step (reverse mode), for checking the
GPU adjoint.

TEST INFRASTRUCTURE (see oracle/__init__.py).

The forward step is restated here with PyTorch CPU tensors in FP64, following
the same literal Table 2 polynomials as hlbm_oracle.c: moments of Eq. 4.5
(u = (j + F/2) / rho, F = rho g), the equilibrium of Eq. 2.2 (3rd order on
D3Q39), the body force of Eq. 3.3, the collision of Eq. 4.4 and periodic
streaming.  torch.autograd then forms exact vector-Jacobian products of one
step at a time over stored forward states, which is the discrete adjoint.
Tests pin this restatement to the C oracle (same states to round-off) and the
gradient to central finite differences of the C oracle.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lattice as _lat


class TorchStep:
    def __init__(self, L: _lat.Lattice, shape, tau_hat: float, thermal: bool = True):
        self.L = L
        self.D = L.D
        self.shape = tuple(shape)
        self.tau = float(tau_hat)
        self.thermal = thermal
        self.c = torch.tensor(L.c, dtype=torch.float64)          # (Q, D)
        self.w = torch.tensor(L.w, dtype=torch.float64)          # (Q,)
        self.cs2 = float(L.cs2)
        self.cc = (self.c ** 2).sum(1)                            # (Q,)
        self.ci = [tuple(int(v) for v in L.c[i]) for i in range(L.Q)]

    def _bc(self, v):  # (Q,) -> (Q, 1, ..., 1)
        return v.view((-1,) + (1,) * len(self.shape))

    def macros(self, f, g):
        rho = f.sum(0)
        j = torch.einsum("qd,q...->d...", self.c, f)
        e = torch.einsum("q,q...->...", self.cc, f)
        F = rho * g
        u = (j + 0.5 * F) / rho
        uu = (u * u).sum(0)
        uF = (u * F).sum(0)
        theta = (e - rho * uu + uF) / (rho * self.D * self.cs2)   # G2 / 2 = u.F
        return rho, u, theta, F

    def collide(self, f, g):
        s, D = self.cs2, self.D
        rho, u, theta, F = self.macros(f, g)
        tb = theta - 1.0 if self.thermal else torch.zeros_like(theta)
        uu = (u * u).sum(0)
        uF = (u * F).sum(0)
        cu = torch.einsum("qd,d...->q...", self.c, u)
        cF = torch.einsum("qd,d...->q...", self.c, F)
        cc = self._bc(self.cc)
        t = (1.0 + cu / s + cu * cu / (2 * s * s) - uu / (2 * s) + tb * (cc - s * D) / (2 * s)
             + cu ** 3 / (6 * s ** 3) - cu * uu / (2 * s * s) + cu * tb * (cc - s * (D + 2)) / (2 * s * s))
        if self.L.feq_order >= 4:
            t = t + (cu ** 4 / (24 * s ** 4) - cu * cu * uu / (4 * s ** 3) + uu * uu / (8 * s * s)
                     + tb * (cu * cu * (cc - s * (D + 4)) + s * uu * (s * (D + 2) - cc)) / (4 * s ** 3)
                     + tb * tb * (cc * cc - 2 * s * (D + 2) * cc + s * s * D * (D + 2)) / (8 * s * s))
        w = self._bc(self.w)
        feq = w * rho * t
        SF = w * (cF / s + cu * cF / (s * s) - uF / s
                  + cF * (cu * cu + tb * s * cc - s * uu - tb * s * s * (D + 2)) / (2 * s ** 3)
                  - cu * uF / (s * s))
        return f - (f - feq) / self.tau + (1.0 - 1.0 / (2.0 * self.tau)) * SF

    def stream(self, fs):
        dims = tuple(range(-1, -self.D - 1, -1))                  # x, y (, z)
        return torch.stack([torch.roll(fs[i], shifts=self.ci[i], dims=dims) for i in range(fs.shape[0])])

    def step(self, f, g):
        return self.stream(self.collide(f, g))

    def kinetic_energy(self, f, g):
        rho, u, _, _ = self.macros(f, g)
        return 0.5 * (rho * (u * u).sum(0)).sum()


def kinetic_energy_gradient(L: _lat.Lattice, shape, tau_hat: float, f0: np.ndarray, g: np.ndarray, steps: int,
                            thermal: bool = True):
    """(L(T), dL/dg) for L = sum rho |u|^2 / 2 after `steps` steps from populations
    f0 [Q, *shape] under the acceleration field g [D, *shape]."""
    ts = TorchStep(L, shape, tau_hat, thermal)
    gt = torch.tensor(np.asarray(g, dtype=np.float64).reshape((L.D,) + tuple(shape)))
    states = [torch.tensor(np.asarray(f0, dtype=np.float64).reshape((L.Q,) + tuple(shape)))]
    with torch.no_grad():
        for _ in range(steps):
            states.append(ts.step(states[-1], gt))
    fT = states[-1].clone().requires_grad_(True)
    gg = gt.clone().requires_grad_(True)
    loss = ts.kinetic_energy(fT, gg)
    lam, dg = torch.autograd.grad(loss, (fT, gg))
    dg = dg.clone()
    for n in range(steps - 1, -1, -1):
        fn = states[n].clone().requires_grad_(True)
        gn = gt.clone().requires_grad_(True)
        out = ts.step(fn, gn)
        lam, dgn = torch.autograd.grad(out, (fn, gn), grad_outputs=lam)
        dg = dg + dgn
    return float(loss.detach()), dg.numpy()
