"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/hlbm.h declares, compiles in the same quadrature the oracle solves
(by an independent solver), and validates its inputs on the host."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import lattice
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    import paper_2411_10751_gb300 as pkg
    pkg.build()
    from paper_2411_10751_gb300 import abi as a
    return a


def _declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(hlbm_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(abi):
    declared = _declared_functions()
    assert declared, "no declarations found"
    lib = C.CDLL(abi.library_path())
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(abi.EXPORTS)


@pytest.mark.parametrize("name,lat", [("D2Q37", 0), ("D3Q39", 1)])
def test_compiled_quadrature_matches_oracle(abi, name, lat):
    L = lattice.get(name)
    c = (C.c_int * (3 * 64))()
    w = (C.c_double * 64)()
    s = C.c_double()
    Q = abi.hlbm_lattice_info(lat, c, w, C.byref(s))
    assert Q == L.Q
    cg = np.array(c[: 3 * Q]).reshape(Q, 3)[:, : L.D]
    wg = np.array(w[:Q])
    assert abs(s.value - L.cs2) < 2e-15   # two independent solves agree to round-off
    # same velocity set (the order is free), same weight per velocity
    ko = {tuple(v): L.w[i] for i, v in enumerate(L.c)}
    assert set(map(tuple, cg)) == set(ko)
    for i in range(Q):
        assert abs(wg[i] - ko[tuple(cg[i])]) < 4e-16 * max(1.0, wg[i] * 1e3)
    # pair order: 2k+1 and 2k+2 are opposite
    for k in range((Q - 1) // 2):
        assert (cg[2 * k + 1] == -cg[2 * k + 2]).all()


def _create(abi, lattice_id=0, nx=16, ny=16, nz=1, tau=0.8, params=None, storage="f32"):
    from paper_2411_10751_gb300.solver import make_params
    p = make_params(params or W.source_params(), storage)
    ctx = C.c_void_p()
    st = abi.hlbm_create(lattice_id, nx, ny, nz, tau, C.byref(p), C.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=6), "HLBM_EINVAL"),
    (dict(ny=3), "HLBM_EINVAL"),
    (dict(nz=2), "HLBM_EINVAL"),
    (dict(tau=0.5), "HLBM_EINVAL"),
    (dict(tau=float("nan")), "HLBM_EINVAL"),
    (dict(params=W.source_params(SC=True)), "HLBM_EINVAL"),                    # SC needs isothermal
    (dict(params=W.source_params(H=True, isothermal=True)), "HLBM_EINVAL"),   # H needs thermal mode
    (dict(params=W.source_params(P=True)), "HLBM_EINVAL"),                     # P needs SC
    (dict(params=W.source_params(H=True, Pr=0.0)), "HLBM_EINVAL"),
    (dict(params=W.source_params(rho0=-1.0)), "HLBM_EINVAL"),
    (dict(lattice_id=1, nz=6), "HLBM_EINVAL"),
    (dict(lattice_id=1, nz=8, params=W.source_params(H=True)), "HLBM_EUNSUPPORTED"),
    (dict(lattice_id=7), "HLBM_EINVAL"),
])
def test_create_rejects_bad_input(abi, kw, expect):
    st, ctx = _create(abi, **kw)
    assert st == getattr(abi, expect)
    assert not ctx.value


def test_create_and_destroy_without_device_work(abi):
    st, ctx = _create(abi, params=W.source_params(force=True, H=True, Pr=0.71))
    assert st == abi.HLBM_OK
    assert abi.hlbm_step_count(ctx) == 0
    assert abi.hlbm_step(ctx, 1) == abi.HLBM_ESTATE          # not initialised
    assert b"hlbm_init" in abi.hlbm_last_error(ctx)
    assert abi.hlbm_set_tile(ctx, 5, 1, 0) == abi.HLBM_EINVAL
    assert abi.hlbm_set_tile(ctx, 4, 2, 0) == abi.HLBM_EINVAL
    assert abi.hlbm_set_tile(ctx, 8, 2, 4) == abi.HLBM_EINVAL
    assert abi.hlbm_set_tile(ctx, 8, 2, 3) == abi.HLBM_OK    # multi-step
    assert abi.hlbm_destroy(ctx) == abi.HLBM_OK


def test_workspace_bytes(abi):
    from paper_2411_10751_gb300.solver import make_params
    p = make_params(W.source_params(force=True), "f32")
    n = abi.hlbm_workspace_bytes(0, 1024, 1024, 1, C.byref(p))
    assert n >= 2 * 37 * 1024 * 1024 * 4 + 2 * 1024 * 1024 * 4
    p16 = make_params(W.source_params(), "f16")
    n16 = abi.hlbm_workspace_bytes(0, 1024, 1024, 1, C.byref(p16))
    assert 2 * 37 * 1024 * 1024 * 2 <= n16 < 2 * 37 * 1024 * 1024 * 4
    assert abi.hlbm_workspace_bytes(0, 3, 3, 1, C.byref(p)) == 0


def test_allocation_failure_is_reported(abi, monkeypatch):
    """Host-side fault injection: the allocator shim fails before any CUDA call."""
    monkeypatch.setenv("HLBM_FAULT_ALLOC", "1")
    st, ctx = _create(abi)
    assert st == abi.HLBM_OK
    r = np.ones(256, np.float32)
    u = np.zeros(512, np.float32)
    assert abi.hlbm_init(ctx, r.ctypes.data, u.ctypes.data, r.ctypes.data, 0) == abi.HLBM_ENOMEM
    assert b"HLBM_FAULT_ALLOC" in abi.hlbm_last_error(ctx)
    abi.hlbm_destroy(ctx)


def test_release_build_has_no_bounds_record(abi):
    """hlbm_debug_record belongs to the bounds-checked build only: the release
    library answers HLBM_EUNSUPPORTED without touching a device."""
    out = (C.c_ulonglong * 4)()
    assert not abi.DEBUG
    assert abi.hlbm_debug_record(out, 1) == abi.HLBM_EUNSUPPORTED
