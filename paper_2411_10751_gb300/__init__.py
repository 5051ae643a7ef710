"""GB300 (sm_103a) implementation of one fused time step of the high-order
BGK lattice Boltzmann method with Hermite body sources (D2Q37 / D3Q39).

The computation lives in libhlbm.so (CUDA kernels behind the C ABI of
include/hlbm.h); ``abi`` binds it with ctypes and ``solver.HLBM`` wraps a
context.  Build the library with ``python -m paper_2411_10751_gb300.build``.
"""
from .build import build  # noqa: F401


def load():
    """Imports the ctypes binding (raises ImportError if libhlbm.so is missing)."""
    from . import abi  # noqa: F401
    from . import solver  # noqa: F401
    return solver
