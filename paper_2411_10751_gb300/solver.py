"""Python front end of the hlbm C ABI: one object per context.

Device memory comes from PyTorch (the context's workspace is a torch uint8
tensor bound with hlbm_bind_memory) and work is ordered on a CUDA stream;
all computation happens in libhlbm's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi

LATTICES = {"D2Q37": abi.HLBM_D2Q37, "D3Q39": abi.HLBM_D3Q39}
STORAGE = {"f32": abi.HLBM_F32, "f16": abi.HLBM_F16, "bf16": abi.HLBM_BF16}
FORCE_KIND = {None: 0, "field": 1, "profile": 2}


def make_params(params: dict, storage: str = "f32") -> abi.hlbm_source_params:
    """hlbm_source_params from a parameter dict (keys as in workloads.source_params)."""
    p = abi.hlbm_source_params()
    flags = 0
    if params.get("force"):
        flags |= abi.HLBM_SRC_FORCE
    if params.get("H"):
        flags |= abi.HLBM_SRC_H
    if params.get("SC"):
        flags |= abi.HLBM_SRC_SC
    if params.get("P"):
        flags |= abi.HLBM_SRC_P
    if params.get("isothermal"):
        flags |= abi.HLBM_ISOTHERMAL
    if params.get("lag"):
        flags |= abi.HLBM_AA     # the in-place step runs the single-pass (lagged) neighbour fields
    if params.get("walls"):
        flags |= abi.HLBM_WALLS
        wu = params.get("wall_u", ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)))
        wt = params.get("wall_theta", (1.0, 1.0))
        for side in range(2):
            v = list(wu[side]) + [0.0, 0.0, 0.0]
            for a in range(3):
                p.wall_u[side][a] = float(v[a])
            p.wall_theta[side] = float(wt[side])
    p.flags = flags
    g = list(params.get("g", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    for a in range(3):
        p.force[a] = float(g[a])
    p.Pr = float(params.get("Pr", 1.0))
    p.eos = {"vdw": 0, "cs": 1}[params.get("eos", "vdw")]
    p.eos_a = float(params.get("eos_a", 0.0))
    p.eos_b = float(params.get("eos_b", 0.0))
    p.eos_T = float(params.get("eos_T", 0.0))
    p.k = float(params.get("k", 0.0))
    p.rho0 = float(params.get("rho0", 1.0))
    p.storage = STORAGE[storage]
    return p


def _dev_f32(x, device) -> torch.Tensor:
    t = torch.as_tensor(x, dtype=torch.float32, device=device)
    return t.contiguous()


class HLBM:
    """A periodic D2Q37 / D3Q39 domain advanced by the fused GPU step."""

    def __init__(self, lattice: str, nx: int, ny: int, nz: int, tau_hat: float, params: dict,
                 storage: str = "f32", device: int | str | torch.device = 0, stream: torch.cuda.Stream | None = None):
        self.lattice, self.nx, self.ny, self.nz = lattice, nx, ny, max(1, nz)
        self.D = 2 if lattice == "D2Q37" else 3
        self.N = nx * ny * self.nz
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.storage = storage
        self._p = make_params(params, storage)
        ctx = C.c_void_p()
        abi.check(abi.hlbm_create(LATTICES[lattice], nx, ny, self.nz, float(tau_hat), C.byref(self._p), C.byref(ctx)))
        self.ctx = ctx
        nbytes = abi.hlbm_workspace_bytes(LATTICES[lattice], nx, ny, self.nz, C.byref(self._p))
        with torch.cuda.device(self.device):
            self._arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            abi.check(abi.hlbm_set_stream(self.ctx, C.c_void_p(s.cuda_stream)), self.ctx)
        abi.check(abi.hlbm_bind_memory(self.ctx, C.c_void_p(self._arena.data_ptr()), nbytes), self.ctx)

    # ------------------------------------------------------------ helpers
    @property
    def shape(self):
        return (self.ny, self.nx) if self.D == 2 else (self.nz, self.ny, self.nx)

    def cuda_stream(self) -> torch.cuda.ExternalStream:
        """The stream the context's kernels run on (for events and ordering)."""
        h = abi.hlbm_get_stream(self.ctx)
        return torch.cuda.ExternalStream(h, device=self.device)

    def _chk(self, st):
        abi.check(st, self.ctx)

    # --------------------------------------------------------------- API
    def init(self, rho, u, theta) -> None:
        """f^ = f^eq(rho, u, theta); torch CUDA tensors stay on the device, anything else is copied from host."""
        if all(isinstance(t, torch.Tensor) and t.is_cuda for t in (rho, u, theta)):
            r, uu, th = (_dev_f32(t, self.device) for t in (rho, u, theta))
            self._chk(abi.hlbm_init(self.ctx, r.data_ptr(), uu.data_ptr(), th.data_ptr(), 1))
            self.synchronize()
        else:
            r, uu, th = (np.ascontiguousarray(np.asarray(t, dtype=np.float32)) for t in (rho, u, theta))
            self._chk(abi.hlbm_init(self.ctx, r.ctypes.data, uu.ctypes.data, th.ctypes.data, 0))

    def set_force_field(self, g, kind: str | None = "field") -> None:
        """Acceleration field: kind 'field' [D, ...], 'profile' [D, ny], or None (uniform params['g'])."""
        if kind is None:
            self._chk(abi.hlbm_set_force_field(self.ctx, None, 0, 0))
            return
        if isinstance(g, torch.Tensor) and g.is_cuda:
            t = _dev_f32(g, self.device)
            self._chk(abi.hlbm_set_force_field(self.ctx, t.data_ptr(), FORCE_KIND[kind], 1))
            self.synchronize()
        else:
            a = np.ascontiguousarray(np.asarray(g, dtype=np.float32))
            self._chk(abi.hlbm_set_force_field(self.ctx, a.ctypes.data, FORCE_KIND[kind], 0))

    def step(self, n: int = 1) -> None:
        self._chk(abi.hlbm_step(self.ctx, int(n)))

    def moments(self):
        """(rho, u, theta) as torch float32 CUDA tensors (ordered on the context's stream)."""
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((self.D,) + self.shape, dtype=torch.float32, device=self.device)
        th = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._chk(abi.hlbm_moments(self.ctx, rho.data_ptr(), u.data_ptr(), th.data_ptr(), 1))
        self.synchronize()
        return rho, u, th

    def moments_host(self):
        """(rho, u, theta) as numpy float32 arrays."""
        rho = np.empty(self.shape, np.float32)
        u = np.empty((self.D,) + self.shape, np.float32)
        th = np.empty(self.shape, np.float32)
        self._chk(abi.hlbm_moments(self.ctx, rho.ctypes.data, u.ctypes.data, th.ctypes.data, 0))
        return rho, u, th

    def diag(self) -> np.ndarray:
        out = (C.c_double * 5)()
        self._chk(abi.hlbm_diag(self.ctx, out))
        return np.array(out[: self.D + 2])

    def save(self) -> bytes:
        n = abi.hlbm_state_bytes(self.ctx)
        buf = C.create_string_buffer(n)
        self._chk(abi.hlbm_save(self.ctx, buf, n))
        return buf.raw

    def load(self, state: bytes) -> None:
        self._chk(abi.hlbm_load(self.ctx, state, len(state)))

    @property
    def step_count(self) -> int:
        return int(abi.hlbm_step_count(self.ctx))

    def set_tile(self, rows: int, nodes_per_thread: int = 0, persistent: int = 0) -> None:
        """Schedule: rows per tile, nodes per thread, persistent (0 default, 1 off, 2 on,
        3 multi-step: one launch for many steps, D2Q37)."""
        self._chk(abi.hlbm_set_tile(self.ctx, int(rows), int(nodes_per_thread), int(persistent)))

    def adjoint(self, steps: int, ckpt_every: int = 50):
        """(L, dL/dg): kinetic energy after `steps` steps from the current state and
        its gradient with respect to the force field (a torch [D, ...] CUDA tensor)."""
        nbytes = abi.hlbm_adjoint_workspace_bytes(self.ctx, int(steps), int(ckpt_every))
        if nbytes == 0:
            raise ValueError("steps and ckpt_every must be >= 1")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        grad = torch.empty((self.D,) + self.shape, dtype=torch.float32, device=self.device)
        loss = C.c_double()
        self._chk(abi.hlbm_adjoint_run(self.ctx, int(steps), int(ckpt_every), C.c_void_p(ws.data_ptr()), nbytes,
                                       C.c_void_p(grad.data_ptr()), C.byref(loss)))
        return loss.value, grad

    def synchronize(self) -> None:
        self._chk(abi.hlbm_synchronize(self.ctx))

    def close(self) -> None:
        if getattr(self, "ctx", None):
            abi.hlbm_destroy(self.ctx)
            self.ctx = None
            self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KineticEnergy(torch.autograd.Function):
    """L(g) = sum rho |u|^2 / 2 after `steps` steps from the initial fields, as a
    differentiable function of the acceleration field g [D, ...]; the gradient
    comes from the adjoint kernels (hlbm_adjoint_run)."""

    @staticmethod
    def forward(ctx, g, solver: "HLBM", rho, u, theta, steps: int, ckpt_every: int = 50):
        solver.init(rho, u, theta)
        solver.set_force_field(g.detach(), "field")
        loss, grad = solver.adjoint(steps, ckpt_every)
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=g.device)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad_out.to(grad.dtype) * grad, None, None, None, None, None, None)


class Batch:
    """Independent periodic D2Q37 domains stepped together (hlbm_batch_*): one
    persistent kernel launch per time step over the tiles of every domain and
    every source kind (graph-replayed)."""

    def __init__(self, solvers: list):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        b = C.c_void_p()
        abi.check(abi.hlbm_batch_create(len(self.solvers), arr, C.byref(b)))
        self.handle = b

    def step(self, n: int = 1) -> None:
        abi.check(abi.hlbm_batch_step(self.handle, int(n)))

    def synchronize(self) -> None:
        abi.check(abi.hlbm_batch_synchronize(self.handle))

    def cuda_stream(self, device=0) -> torch.cuda.ExternalStream:
        return torch.cuda.ExternalStream(abi.hlbm_batch_get_stream(self.handle), device=device)

    def close(self) -> None:
        if getattr(self, "handle", None):
            abi.hlbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
