"""Multi-step persistent D2Q37 kernel (hlbm_set_tile(rows, npt, 3)).

One launch runs many steps; the tile of step s starts once its 3 x 3
neighbourhood of step s - 1 has been stored (per-tile completion flags).  The
arithmetic per node is that of the one-launch-per-step kernels, so the saved
populations must agree bit for bit with the persistent kernel's, over launch
boundaries (split step calls, odd step counts) and with the TMA path off;
against the FP64 oracle the FP32 bar of the parity tests holds.
"""
import numpy as np
import pytest

import workloads as W
from oracle.solver import Oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def HLBM():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300.solver import HLBM as cls
    return cls


def _case(kind, nx, ny):
    if kind == "thermal":
        return W.thermal_decay(nx=nx, ny=ny, tau_hat=0.7, Pr=0.71)
    if kind == "kolmogorov":
        return W.kolmogorov(nx=nx, ny=ny)
    return W.droplet(nx=nx, ny=ny, r0=0.25 * min(nx, ny), k=1.5672)


def _run(HLBM, c, schedule, chunks, storage="f32"):
    g = HLBM(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params, storage=storage)
    g.set_tile(*schedule)
    if c.gfield is not None:
        g.set_force_field(c.gfield, "field")
    g.init(c.rho, c.u, c.theta)
    for n in chunks:
        g.step(n)
    state = g.save()
    m = g.moments_host()
    assert g.step_count == sum(chunks)
    g.close()
    return state, m


def _rel_err(m_gpu, m_ora):
    (rho, u, th), (r0, u0, t0) = m_gpu, m_ora
    er = np.abs(rho - r0).max() / np.abs(r0).max()
    eu = np.sqrt(((u - u0) ** 2).sum(0)).max() / max(np.sqrt((u0 ** 2).sum(0)).max(), 1e-300)
    et = np.abs(th - t0).max() / np.abs(t0).max()
    return er, eu, et


@pytest.mark.parametrize("kind,nx,ny,rows,npt", [
    ("thermal", 128, 96, 8, 2), ("thermal", 64, 40, 4, 1), ("thermal", 96, 64, 16, 2),
    ("kolmogorov", 64, 64, 8, 2), ("droplet", 96, 64, 8, 1), ("droplet", 64, 48, 16, 2)])
def test_multistep_equals_per_step_launches(HLBM, kind, nx, ny, rows, npt):
    """Bit-identical populations after 61 steps taken as 7 + 33 + 21 (three
    multi-step launches, odd lengths) and as 61 single-step persistent launches."""
    c = _case(kind, nx, ny)
    ref, _ = _run(HLBM, c, (rows, npt, 2), [61])
    got, _ = _run(HLBM, c, (rows, npt, 3), [7, 33, 21])
    assert got == ref


def test_multistep_without_tma(HLBM, monkeypatch):
    """With the TMA path off every tile is filled by L2 loads of the other
    CTAs' results: still bit-identical."""
    c = _case("thermal", 128, 64)
    ref, _ = _run(HLBM, c, (8, 2, 2), [40])
    monkeypatch.setenv("HLBM_NO_TMA", "1")
    got, _ = _run(HLBM, c, (8, 2, 3), [40])
    assert got == ref


@pytest.mark.parametrize("kind", ["thermal", "kolmogorov", "droplet"])
def test_multistep_oracle_parity(HLBM, kind):
    c = _case(kind, 128, 96)
    _, mg = _run(HLBM, c, (8, 2, 3), [100])
    o = Oracle(c.lattice, c.nx, c.ny, c.nz, c.tau_hat, c.params)
    if c.gfield is not None:
        o.set_force_field(c.gfield)
    o.init(c.rho, c.u, c.theta)
    o.run(100)
    err = _rel_err(mg, o.moments())
    assert max(err) < TOL32, err


def test_multistep_thermal_1024(HLBM):
    """The benchmark workload at full size, multi-step schedule, against the
    per-step persistent kernel (bit for bit) after 100 steps."""
    c = W.thermal_decay(n=1024)
    ref, _ = _run(HLBM, c, (8, 2, 2), [100])
    got, _ = _run(HLBM, c, (8, 2, 3), [100])
    assert got == ref


def test_multistep_falls_back_on_ragged_domains(HLBM):
    """Domains the tiles do not cover exactly run the per-step kernels."""
    c = _case("thermal", 100, 75)
    ref, _ = _run(HLBM, c, (8, 2, 2), [30])
    got, _ = _run(HLBM, c, (8, 2, 3), [30])
    assert got == ref


@pytest.mark.parametrize("lattice", ["D2Q37", "D3Q39"])
def test_persistent_equals_one_cta_per_tile(HLBM, lattice):
    """The persistent kernels (prefetch, tile order reversed every other step,
    D3Q39: whole-row tiles with the force field staged by TMA) run the same
    per-node arithmetic as the one-CTA-per-tile kernels: bit-identical states
    after an odd number of steps."""
    if lattice == "D2Q37":
        c = _case("thermal", 128, 96)
    else:
        c = W.taylor_green_3d(n=64, tau_hat=0.7, Ma=0.2)
        sl = (slice(0, 13), slice(0, 19), slice(0, 64))
        c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
        c.u = c.u[(slice(None),) + sl].copy()
        c.nz, c.ny, c.nx = c.rho.shape
        rng = np.random.default_rng(3)
        c.gfield = W.fp32(2e-5 * (2 * rng.random((3,) + c.rho.shape) - 1))
    ref, _ = _run(HLBM, c, (8, 2, 1), [37])
    got, _ = _run(HLBM, c, (8, 2, 2), [37])
    assert got == ref
