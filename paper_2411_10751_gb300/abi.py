"""ctypes binding of libhlbm.so, one Python function per C entry point of
include/hlbm.h, with the same names and argument order.  Argument marshalling
only: every step of the computation runs in the library's CUDA kernels.

Importing this module loads the in-tree library
(paper_2411_10751_gb300/_build/libhlbm.so; with the environment variable
HLBM_LIBRARY=debug its bounds-checking variant _build/debug/libhlbm_debug.so)
and raises ImportError if it has not been built; there is no fallback
implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

_BUILD = Path(__file__).resolve().parent / "_build"
DEBUG = os.environ.get("HLBM_LIBRARY", "") == "debug"
LIB_PATH = _BUILD / "debug" / "libhlbm_debug.so" if DEBUG else _BUILD / "libhlbm.so"

HLBM_D2Q37, HLBM_D3Q39 = 0, 1
HLBM_F32, HLBM_F16, HLBM_BF16 = 0, 1, 2
HLBM_SRC_FORCE, HLBM_SRC_H, HLBM_SRC_SC, HLBM_SRC_P, HLBM_ISOTHERMAL, HLBM_WALLS, HLBM_AA = 1, 2, 4, 8, 16, 32, 64
STATUS = {0: "HLBM_OK", 1: "HLBM_EINVAL", 2: "HLBM_ENOMEM", 3: "HLBM_ECUDA", 4: "HLBM_EDIVERGED",
          5: "HLBM_ETIMEOUT", 6: "HLBM_ESTATE", 7: "HLBM_EUNSUPPORTED"}
for _k, _v in STATUS.items():
    globals()[_v] = _k

# every symbol include/hlbm.h declares
EXPORTS = ["hlbm_workspace_bytes", "hlbm_create", "hlbm_bind_memory", "hlbm_set_stream", "hlbm_get_stream",
           "hlbm_init", "hlbm_set_force_field", "hlbm_step", "hlbm_moments", "hlbm_diag", "hlbm_state_bytes",
           "hlbm_save", "hlbm_load", "hlbm_step_count", "hlbm_set_tile", "hlbm_synchronize", "hlbm_set_wait_timeout",
           "hlbm_last_error", "hlbm_destroy", "hlbm_lattice_info", "hlbm_population_sums_noalloc",
           "hlbm_adjoint_workspace_bytes", "hlbm_adjoint_run", "hlbm_batch_create", "hlbm_batch_step",
           "hlbm_batch_synchronize", "hlbm_batch_get_stream", "hlbm_batch_destroy", "hlbm_debug_record"]


class hlbm_source_params(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("force", C.c_double * 3), ("Pr", C.c_double), ("eos", C.c_int),
                ("eos_a", C.c_double), ("eos_b", C.c_double), ("eos_T", C.c_double), ("k", C.c_double),
                ("rho0", C.c_double), ("storage", C.c_int), ("wall_u", (C.c_double * 3) * 2),
                ("wall_theta", C.c_double * 2)]


class HLBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


if not LIB_PATH.exists():
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2411_10751_gb300.build"
                      f"{' --debug' if DEBUG else ''}` (or __graft_entry__.build())")

_lib = C.CDLL(str(LIB_PATH))

_vp, _i, _d, _sz, _ll = C.c_void_p, C.c_int, C.c_double, C.c_size_t, C.c_longlong
_P = C.POINTER(hlbm_source_params)
_sigs = {
    "hlbm_workspace_bytes": ([_i, _i, _i, _i, _P], _sz),
    "hlbm_create": ([_i, _i, _i, _i, _d, _P, C.POINTER(_vp)], _i),
    "hlbm_bind_memory": ([_vp, _vp, _sz], _i),
    "hlbm_set_stream": ([_vp, _vp], _i),
    "hlbm_get_stream": ([_vp], _vp),
    "hlbm_init": ([_vp, _vp, _vp, _vp, _i], _i),
    "hlbm_set_force_field": ([_vp, _vp, _i, _i], _i),
    "hlbm_step": ([_vp, _i], _i),
    "hlbm_moments": ([_vp, _vp, _vp, _vp, _i], _i),
    "hlbm_diag": ([_vp, C.POINTER(C.c_double)], _i),
    "hlbm_state_bytes": ([_vp], _sz),
    "hlbm_save": ([_vp, _vp, _sz], _i),
    "hlbm_load": ([_vp, _vp, _sz], _i),
    "hlbm_step_count": ([_vp], _ll),
    "hlbm_set_tile": ([_vp, _i, _i, _i], _i),
    "hlbm_synchronize": ([_vp], _i),
    "hlbm_set_wait_timeout": ([_vp, _d], _i),
    "hlbm_last_error": ([_vp], C.c_char_p),
    "hlbm_destroy": ([_vp], _i),
    "hlbm_lattice_info": ([_i, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)], _i),
    "hlbm_population_sums_noalloc": ([_i, _ll, _i, _d, _vp, _vp, C.POINTER(C.c_double)], _i),
    "hlbm_adjoint_workspace_bytes": ([_vp, _i, _i], _sz),
    "hlbm_adjoint_run": ([_vp, _i, _i, _vp, _sz, _vp, C.POINTER(C.c_double)], _i),
    "hlbm_batch_create": ([_i, C.POINTER(_vp), C.POINTER(_vp)], _i),
    "hlbm_batch_step": ([_vp, _i], _i),
    "hlbm_batch_synchronize": ([_vp], _i),
    "hlbm_batch_get_stream": ([_vp], _vp),
    "hlbm_batch_destroy": ([_vp], _i),
    "hlbm_debug_record": ([C.POINTER(C.c_ulonglong), _i], _i),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f


def check(status: int, ctx=None) -> None:
    """Raise HLBMError for a non-OK status, with the context's message."""
    if status != HLBM_OK:
        msg = hlbm_last_error(ctx).decode() if ctx else ""
        raise HLBMError(status, msg)


def library_path() -> str:
    return str(LIB_PATH)


def debug_record(clear: bool = True):
    """The debug library's bounds record: (count, site, index, bound) of the
    first rejected access on the current device (zeros: none)."""
    out = (C.c_ulonglong * 4)()
    check(hlbm_debug_record(out, int(clear)))
    return tuple(int(v) for v in out)
