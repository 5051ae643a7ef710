"""GPU parity: the CUDA fused step (through the C ABI) against the FP64 oracle.

Metric (per field q in rho, u, theta): max over nodes of |q_gpu - q_oracle|
divided by max |q_oracle| (|.| the vector norm for u).  Bar for FP32
storage: 1e-5 after 100 steps.  Reduced-precision storage: max|u - u_oracle|
/ max|u| <= 1e-3 (FP16).
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


def rel_err(m_gpu, m_ora):
    rho, u, th = m_gpu
    r0, u0, t0 = m_ora
    er = np.abs(rho - r0).max() / np.abs(r0).max()
    eu = np.sqrt(((u - u0) ** 2).sum(0)).max() / max(np.sqrt((u0 ** 2).sum(0)).max(), 1e-300)
    et = np.abs(th - t0).max() / np.abs(t0).max()
    return er, eu, et


def run_pair(HLBM, case, steps, storage="f32", rows=None, force_kind="field", npt=0, persistent=0):
    g = HLBM(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params, storage=storage)
    if rows:
        g.set_tile(rows, npt, persistent)
    o = Oracle(case.lattice, case.nx, case.ny, case.nz, case.tau_hat, case.params)
    if case.gfield is not None:
        o.set_force_field(case.gfield)
        if force_kind == "profile":
            g.set_force_field(case.gfield[:, :, 0] if case.D == 2 else case.gfield[:, 0, :, 0], "profile")
        else:
            g.set_force_field(case.gfield, "field")
    g.init(case.rho, case.u, case.theta)
    o.init(case.rho, case.u, case.theta)
    g.step(steps)
    o.run(steps)
    mg = g.moments_host()
    mo = o.moments()
    g.close()
    return mg, mo


def test_kolmogorov_64_parity_and_profile(HLBM):
    c = W.kolmogorov(64)
    mg, mo = run_pair(HLBM, c, 100)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


def test_kolmogorov_64_2000_steps(HLBM):
    from oracle import analytic, lattice
    c = W.kolmogorov(64)
    mg, mo = run_pair(HLBM, c, 2000, force_kind="profile")
    assert max(rel_err(mg, mo)) < 1e-4, rel_err(mg, mo)
    nu = analytic.viscosity(lattice.d2q37().cs2, c.tau_hat)
    ua = analytic.kolmogorov_ux(np.arange(64), 2000, c.meta["g0"], nu, 64)
    assert np.abs(mg[1][0] - ua[:, None]).max() / np.abs(ua).max() < 1e-2


# On 7 x 7 the sin(2 pi y / 7) shear mode decays by exp(-nu k^2 t) = e^-11 in
# 100 steps, leaving u at FP32 noise; 10 steps keep the signal.
@pytest.mark.parametrize("nx,ny,steps", [(7, 7, 10), (45, 37, 100), (100, 75, 100)])
def test_thermal_parity_ragged(HLBM, nx, ny, steps):
    c = W.thermal_decay(nx=nx, ny=ny, tau_hat=0.7, Pr=0.71)
    mg, mo = run_pair(HLBM, c, steps)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


# (rows, nodes per thread, persistent: 1 off / 2 on)
SCHEDULES = [(4, 1, 1), (8, 1, 1), (8, 2, 1), (16, 1, 1), (16, 2, 1), (4, 1, 2), (8, 1, 2), (8, 2, 2), (16, 2, 2)]


@pytest.mark.parametrize("rows,npt,pers", SCHEDULES)
def test_thermal_schedules(HLBM, rows, npt, pers):
    # 200 x 120: interior tiles take the TMA path, edge tiles the gather path
    c = W.thermal_decay(nx=200, ny=120, tau_hat=0.7, Pr=0.71)
    mg, mo = run_pair(HLBM, c, 30, rows=rows, npt=npt, persistent=pers)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("rows,npt,pers", SCHEDULES)
def test_droplet_schedules(HLBM, rows, npt, pers):
    c = W.droplet(nx=160, ny=96, r0=25.0, k=1.5672)
    mg, mo = run_pair(HLBM, c, 30, rows=rows, npt=npt, persistent=pers)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("rows,npt,pers", SCHEDULES)
def test_kolmogorov_schedules(HLBM, rows, npt, pers):
    c = W.kolmogorov(nx=160, ny=96)
    mg, mo = run_pair(HLBM, c, 30, rows=rows, npt=npt, force_kind="profile", persistent=pers)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("pers", [1, 2])
@pytest.mark.parametrize("kind,nx,ny", [("thermal", 8, 12), ("thermal", 36, 20), ("droplet", 32, 32),
                                        ("droplet", 40, 28)])
def test_domains_narrower_than_a_staged_row(HLBM, kind, nx, ny, pers):
    """Domains narrower than a staged box row: each row wraps several times;
    with persistent CTAs (pers 2) most CTAs draw a stop index at once."""
    if kind == "thermal":
        c = W.thermal_decay(nx=nx, ny=ny, tau_hat=0.7, Pr=0.71)
    else:
        c = W.droplet(nx=nx, ny=ny, r0=0.25 * nx, k=1.5672)
    mg, mo = run_pair(HLBM, c, 30, rows=8, npt=2, persistent=pers)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


def test_thermal_1024_full_size(HLBM):
    """The benchmark workload at its full size on the default schedule (one CTA
    per tile); the schedules the benchmark times at this size are checked in
    test_gpu_fullsize.py."""
    c = W.thermal_decay(n=1024)
    mg, mo = run_pair(HLBM, c, 100)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("k", [0.01, 1.5672])
def test_droplet_parity_small(HLBM, k):
    c = W.droplet(nx=70, ny=53, r0=14.0, k=k)
    mg, mo = run_pair(HLBM, c, 100)
    er, eu, et = rel_err(mg, mo)
    assert er < TOL32 and et < TOL32 and eu < TOL32, (er, eu, et)


def test_droplet_512_full_size(HLBM):
    c = W.droplet(n=512)
    mg, mo = run_pair(HLBM, c, 100)
    er, eu, et = rel_err(mg, mo)
    assert er < TOL32 and et < TOL32 and eu < TOL32, (er, eu, et)


@pytest.mark.parametrize("Tr", [0.7, 0.9])
def test_carnahan_starling_droplet_parity(HLBM, Tr):
    """Carnahan-Starling droplet as printed for Sec. 5.4 (a = 0.25, b = 4,
    k = 3.02; 200 x 200, r0 = 50)."""
    c = W.droplet(n=200, r0=50.0, Tr=Tr, k=3.02, eos="cs")
    mg, mo = run_pair(HLBM, c, 100)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


def test_d3q39_taylor_green_parity(HLBM):
    c = W.taylor_green_3d(n=16, tau_hat=0.6, Ma=0.3)
    rng = np.random.default_rng(0)
    c.gfield = W.fp32(1e-5 * (2 * rng.random(c.gfield.shape) - 1))
    mg, mo = run_pair(HLBM, c, 50)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("rows,npt,pers,nx", [(4, 1, 1, 22), (8, 1, 1, 22), (8, 2, 1, 22), (8, 2, 2, 22),
                                               (8, 2, 2, 32), (8, 2, 2, 64)])
def test_d3q39_schedules(HLBM, rows, npt, pers, nx):
    """Every D3Q39 tile shape (one node per thread, two on paired lanes, and the
    persistent whole-row kernel, which serves nx = 32 and 64 here and falls back
    to the grid kernel at nx = 22) on a ragged box with a full acceleration field."""
    c = W.taylor_green_3d(n=64, tau_hat=0.7, Ma=0.2)
    sl = (slice(0, 13), slice(0, 19), slice(0, nx))
    c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
    c.u = c.u[(slice(None),) + sl].copy()
    c.nz, c.ny, c.nx = c.rho.shape
    rng = np.random.default_rng(3)
    c.gfield = W.fp32(2e-5 * (2 * rng.random((3,) + c.rho.shape) - 1))
    mg, mo = run_pair(HLBM, c, 30, rows=rows, npt=npt, persistent=pers)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


def test_d3q39_ragged_uniform_force(HLBM):
    c = W.taylor_green_3d(n=24, tau_hat=0.7, Ma=0.1)
    # ragged non-cubic 21 x 11 x 9 box: crop the fields
    sl = (slice(0, 9), slice(0, 11), slice(0, 21))
    c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
    c.u = c.u[(slice(None),) + sl].copy()
    c.nz, c.ny, c.nx = c.rho.shape
    c.gfield = None
    c.params["g"] = (1e-5, -2e-5, 3e-5)
    mg, mo = run_pair(HLBM, c, 40)
    assert max(rel_err(mg, mo)) < TOL32, rel_err(mg, mo)


@pytest.mark.parametrize("storage,tol_u", [("f16", 1e-3), ("bf16", 2e-2)])
def test_reduced_precision_storage(HLBM, storage, tol_u):
    c = W.thermal_decay(nx=128, ny=128, tau_hat=0.7, Pr=0.71)
    mg, mo = run_pair(HLBM, c, 100, storage=storage)
    er, eu, et = rel_err(mg, mo)
    assert eu < tol_u, (storage, er, eu, et)


@pytest.mark.parametrize("storage,nx", [("f16", 32), ("f16", 64), ("bf16", 64)])
def test_d3q39_reduced_precision_rows(HLBM, storage, nx):
    """16-bit storage on D3Q39: at nx = 32 a stored row is 64 bytes and the
    step runs the grid kernel; at nx = 64 the persistent whole-row kernel,
    with the y-edge planes copied row by row (ny = 19 is not a multiple of
    the 4-row tiles).  Against the FP64 oracle within the storage bars."""
    c = W.taylor_green_3d(n=64, tau_hat=0.7, Ma=0.2)
    sl = (slice(0, 13), slice(0, 19), slice(0, nx))
    c.rho, c.theta = c.rho[sl].copy(), c.theta[sl].copy()
    c.u = c.u[(slice(None),) + sl].copy()
    c.nz, c.ny, c.nx = c.rho.shape
    rng = np.random.default_rng(3)
    c.gfield = W.fp32(2e-5 * (2 * rng.random((3,) + c.rho.shape) - 1))
    mg, mo = run_pair(HLBM, c, 30, storage=storage, rows=8, npt=2, persistent=2)
    er, eu, et = rel_err(mg, mo)
    assert eu < (1e-3 if storage == "f16" else 2e-2), (storage, er, eu, et)


def test_force_profile_equals_full_field_bitwise(HLBM):
    c = W.kolmogorov(64, nx=40, ny=50)
    a, _ = run_pair(HLBM, c, 30, force_kind="field")
    b, _ = run_pair(HLBM, c, 30, force_kind="profile")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_graph_replay_equals_single_steps_bitwise(HLBM):
    c = W.thermal_decay(nx=48, ny=40, tau_hat=0.7, Pr=0.71)
    g1 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g2 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g1.init(c.rho, c.u, c.theta)
    g2.init(c.rho, c.u, c.theta)
    g1.step(70)                      # two graph replays of 32 steps + 6 single steps
    for _ in range(70):
        g2.step(1)
    for x, y in zip(g1.moments_host(), g2.moments_host()):
        assert np.array_equal(x, y)
    assert g1.step_count == g2.step_count == 70


def test_save_load_resume_bitwise(HLBM):
    c = W.droplet(nx=48, ny=40, r0=10.0, k=1.0)
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g.init(c.rho, c.u, c.theta)
    g.step(100)
    ref = g.moments_host()
    g.init(c.rho, c.u, c.theta)
    g.step(60)
    state = g.save()
    g2 = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g2.load(state)
    assert g2.step_count == 60
    g2.step(40)
    for x, y in zip(ref, g2.moments_host()):
        assert np.array_equal(x, y)


def test_fp64_diagnostics_conservation(HLBM):
    rho = 1.0 + 0.02 * np.sin(2 * np.pi * np.arange(40) / 40)[None, :] * np.ones((36, 1))
    u = np.zeros((2, 36, 40))
    u[0] = 0.01 * np.cos(2 * np.pi * np.arange(36) / 36)[:, None]
    th = 1.0 + 0.01 * np.cos(2 * np.pi * np.arange(40) / 40)[None, :] * np.ones((36, 1))
    p = W.source_params(H=True, Pr=0.71)
    g = HLBM("D2Q37", 40, 36, 1, 0.7, p)
    o = Oracle("D2Q37", 40, 36, 1, 0.7, p)
    g.init(rho, u, th)
    o.init(rho, u, th)
    d0 = g.diag()
    g.step(500)
    o.run(500)
    d1 = g.diag()
    do = o.diag()
    assert abs(d1[0] - d0[0]) < 1e-6 * d0[0]               # FP32 storage, FP64 sums
    assert np.abs(d1[1:3] - d0[1:3]).max() < 1e-6 * d0[0]
    assert abs(d1[3] - d0[3]) < 1e-6 * d0[3]
    assert np.abs(d1 - do).max() < 1e-5 * np.abs(do).max()


def test_divergence_is_detected_and_sticky(HLBM):
    from paper_2411_10751_gb300 import abi
    c = W.thermal_decay(nx=32, ny=32)
    rho = c.rho.copy()
    rho[5, 7] = np.nan               # a non-finite state must be reported, not hidden
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g.init(rho, c.u, c.theta)
    g.step(2)
    with pytest.raises(abi.HLBMError) as e:
        g.diag()
    assert e.value.status == abi.HLBM_EDIVERGED
    with pytest.raises(abi.HLBMError) as e2:
        g.step(1)
    assert e2.value.status == abi.HLBM_ESTATE
    g.init(c.rho, c.u, c.theta)      # a fresh init clears the error state
    g.step(1)
    assert np.isfinite(g.diag()).all()


def test_zero_steps_is_identity(HLBM):
    c = W.kolmogorov(16)
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    g.init(c.rho, c.u, c.theta)
    a = g.moments_host()
    g.step(0)
    b = g.moments_host()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.abs(a[0] - 1.0).max() < 1e-7


def test_expired_device_wait_reports_timeout(HLBM, monkeypatch):
    """A TMA-staged tile whose barrier is armed but never receives its copies
    (test hook) must give up after the wall-time limit, report HLBM_ETIMEOUT
    through the status word, and leave the device usable."""
    from paper_2411_10751_gb300 import abi
    c = W.thermal_decay(n=256)
    monkeypatch.setenv("HLBM_TEST_SKIP_TMA", "1")
    g = HLBM(c.lattice, c.nx, c.ny, 1, c.tau_hat, c.params)
    monkeypatch.delenv("HLBM_TEST_SKIP_TMA")
    abi.check(abi.hlbm_set_wait_timeout(g.ctx, 0.01), g.ctx)
    g.init(c.rho, c.u, c.theta)
    g.step(1)
    with pytest.raises(abi.HLBMError) as e:
        g.synchronize()
    assert e.value.status == abi.HLBM_ETIMEOUT
    g.close()
    # the device and a new context keep working
    mg, mo = run_pair(HLBM, c, 10)
    assert max(rel_err(mg, mo)) < TOL32
