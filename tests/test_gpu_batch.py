"""Batched step (hlbm_batch_*) on the GPU.

1. Each domain of a mixed batch (Kolmogorov with H_i, vdW droplets, a plain
   body-force domain; uneven sizes and parameters) matches the FP64 oracle.
2. A batch step equals stepping every context on its own, bit for bit (both
   run the same tile code).
3. The full workload: 256 domains of sides 32..256 (about 6.4 M nodes), 100
   steps in graph-replayed batch launches; sampled domains against the oracle.
"""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Oracle

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300 import solver
    return solver


def _ctx(lib, c):
    g = lib.HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    if c.gfield is not None:
        g.set_force_field(c.gfield[:, :, 0], "profile")
    g.init(c.rho, c.u, c.theta)
    return g


def _oracle(c, steps):
    o = Oracle(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    if c.gfield is not None:
        o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    o.run(steps)
    return o.moments()


def _err(mg, mo):
    r, u, t = mg
    r0, u0, t0 = mo
    return (np.abs(r - r0).max() / np.abs(r0).max(),
            np.sqrt(((u - u0) ** 2).sum(0)).max() / np.sqrt((u0 ** 2).sum(0)).max(),
            np.abs(t - t0).max() / np.abs(t0).max())


def _mixed_cases():
    cases = W.batched(10, seed=3, nmin=32, nmax=90)
    plain = W.kolmogorov(nx=45, ny=38)      # body force only
    return cases + [plain]


def test_batch_domains_match_oracle(lib):
    cases = _mixed_cases()
    ctxs = [_ctx(lib, c) for c in cases]
    b = lib.Batch(ctxs)
    b.step(60)
    b.synchronize()
    for c, g in zip(cases, ctxs):
        e = _err(g.moments_host(), _oracle(c, 60))
        assert max(e) < TOL32, (c.name, c.nx, e)
        assert g.step_count == 60
    b.close()


def test_batch_equals_individual_steps_bitwise(lib):
    cases = _mixed_cases()
    batched = [_ctx(lib, c) for c in cases]
    single = [_ctx(lib, c) for c in cases]
    b = lib.Batch(batched)
    b.step(7)               # three graph replays of two steps and one single launch
    b.synchronize()
    for s in single:
        s.step(7)
    for x, y in zip(batched, single):
        for p, q in zip(x.moments_host(), y.moments_host()):
            assert np.array_equal(p, q)
    b.close()


def test_full_batched_workload(lib):
    cases = W.batched(256, seed=0)
    ctxs = [_ctx(lib, c) for c in cases]
    b = lib.Batch(ctxs)
    b.step(100)
    b.synchronize()
    sizes = np.array([c.nodes for c in cases])
    sample = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 0, 1, 101, 202, 255})
    for k in sample:
        e = _err(ctxs[k].moments_host(), _oracle(cases[k], 100))
        assert max(e) < TOL32, (k, cases[k].name, cases[k].nx, e)
    for g in ctxs:
        assert np.isfinite(g.diag()).all()
    b.close()
