"""Small runs over every kernel family of the library, for the bounds-checked
debug build (test_gpu_debug_build.py).  Run as a script it loads the library
that HLBM_LIBRARY selects, runs every case and writes the results and the
library's bounds record after each case to an .npz file:

    HLBM_LIBRARY=debug python tests/debug_cases.py out.npz

Each case is small, yet large enough that its launch shapes take their
multi-tile paths (persistent CTAs with several tiles each, edge tiles with
wrapped gathers, ragged rows and columns, TMA-staged interior tiles).
"""
from __future__ import annotations

import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import workloads as W  # noqa: E402


def _lagged(c):
    c.params = dict(c.params)
    c.params["lag"] = True
    return c


def _force3d(c, amp=2e-4, seed=5):
    rng = np.random.default_rng(seed)
    c.gfield = W.fp32(amp * (2 * rng.random((3,) + c.rho.shape) - 1))
    c.params = dict(c.params)
    c.params["force"] = True
    return c


def _run(HLBM, c, steps, sched=None, storage="f32", field_kind=None):
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=storage)
    if sched:
        g.set_tile(*sched)
    if c.gfield is not None:
        g.set_force_field(c.gfield, field_kind or "field")
    g.init(c.rho, c.u, c.theta)
    g.step(steps)
    out = [x.astype(np.float32) for x in g.moments_host()]
    g.close()
    return out


def cases():
    """name -> callable(solver module) returning a list of arrays."""
    def thermal_persistent(S):          # 1,024 tiles on 456 CTAs: the prefetch path
        return _run(S.HLBM, W.thermal_decay(n=512), 12, (8, 2, 2))

    def thermal_multistep(S):           # one launch for many steps
        return _run(S.HLBM, W.thermal_decay(n=512), 40, (8, 2, 3))

    def thermal_ragged(S):              # edge tiles, ragged rows and columns, TMA stores
        return _run(S.HLBM, W.thermal_decay(nx=200, ny=122), 12)

    def thermal_f16(S):
        return _run(S.HLBM, W.thermal_decay(n=256), 12, (8, 2, 2), storage="f16")

    def droplet(S):                     # psi on the three-node frame
        return _run(S.HLBM, W.droplet(n=160, r0=30.0), 12, (8, 1, 2))

    def kolmogorov_profile(S):          # body force from a y profile
        c = W.kolmogorov(nx=96, ny=80, g0=1e-4)
        c.gfield = c.gfield[:, :, 0].copy()
        return _run(S.HLBM, c, 12, field_kind="profile")

    def walls(S):
        return _run(S.HLBM, W.rayleigh_benard(nx=64, ny=34, Ra=8000.0, roll=0.01), 12)

    def in_place_odd(S):                # in-place streaming, odd step count
        return _run(S.HLBM, _lagged(W.thermal_decay(nx=200, ny=122)), 13)

    def in_place_droplet(S):
        return _run(S.HLBM, _lagged(W.droplet(n=96, r0=20.0)), 12)

    def d3q39_gather(S):                # row-tile kernel on a domain of odd sizes
        f = W.random_small("D3Q39", nx=13, ny=19, nz=11, seed=4, amp_u=0.02, amp_T=0.02, amp_rho=0.02)
        c = W.Case("random3d", "D3Q39", 13, 19, 11, 0.7, W.source_params(force=True), f["rho"], f["u"], f["theta"])
        return _run(S.HLBM, _force3d(c), 8)

    def d3q39_rows(S):                  # whole-row persistent kernel, staged force field
        c = _force3d(W.taylor_green_3d(n=64, tau_hat=0.6, Ma=0.1))
        return _run(S.HLBM, c, 6, (8, 2, 2))

    def batch(S):
        cs = W.batched(6, seed=3, nmin=32, nmax=90)
        ctx = []
        for c in cs:
            g = S.HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
            if c.gfield is not None:
                g.set_force_field(c.gfield[:, :, 0], "profile")
            g.init(c.rho, c.u, c.theta)
            ctx.append(g)
        b = S.Batch(ctx)
        b.step(10)
        b.synchronize()
        out = [x.astype(np.float32) for g in ctx for x in g.moments_host()]
        b.close()
        for g in ctx:
            g.close()
        return out

    def adjoint(S):                     # reverse rows kernel, checkpoint segments
        c = _force3d(W.taylor_green_3d(n=32, tau_hat=0.6, Ma=0.1))
        g = S.HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
        g.set_force_field(c.gfield, "field")
        g.init(c.rho, c.u, c.theta)
        loss, grad = g.adjoint(6, 4)
        out = [np.array([loss]), grad.cpu().numpy()]
        g.close()
        return out

    return {k: v for k, v in locals().items() if callable(v)}


def main(path: str) -> None:
    from paper_2411_10751_gb300 import abi, solver
    res = {"debug": np.array([abi.DEBUG])}
    for name, fn in cases().items():
        print(name, flush=True)
        arrs = fn(solver)
        for k, a in enumerate(arrs):
            res[f"{name}/{k}"] = np.asarray(a)
        res[f"{name}/record"] = np.array(abi.debug_record(clear=True) if abi.DEBUG else (0, 0, 0, 0),
                                         dtype=np.uint64)
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
