"""Convenience wrapper over the C ABI: one ``Solver`` per ndg_ctx.

Torch supplies the device memory of the caller's arrays and the CUDA stream the context runs on;
all computation is libndg's.  Arrays use the element layout U[v][e][node] (``shape``).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import native as nat

DTYPES = {"f64": (nat.NDG_F64, torch.float64, np.float64), "f32": (nat.NDG_F32, torch.float32, np.float32),
          "f64ff": (nat.NDG_F64_FF, torch.float64, np.float64)}


class Solver:
    def __init__(self, dim: int, degree: int, elems, equation: int = nat.NDG_ADVECTION,
                 flux: int | None = None, dtype: str = "f64", length=(1.0, 1.0, 1.0),
                 velocity=(1.0, 0.0, 0.0), sound_speed: float = 1.0, elems_per_block: int = 0,
                 device: int = 0, stream: torch.cuda.Stream | None = None, kernel: int = 0,
                 mass: int = 0):
        if flux is None:
            flux = nat.NDG_FLUX_UPWIND if equation == nat.NDG_ADVECTION else nat.NDG_FLUX_LLF
        self.dtype_code, self.torch_dtype, self.np_dtype = DTYPES[dtype]
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        cfg = nat.ndg_config_init()
        cfg.dim, cfg.degree = dim, degree
        e = list(elems) if hasattr(elems, "__len__") else [elems] * dim
        for a in range(3):
            cfg.elems[a] = e[a] if a < dim else 1
            cfg.length[a] = length[a] if a < len(length) else 1.0
            cfg.velocity[a] = velocity[a] if a < len(velocity) else 0.0
        cfg.equation, cfg.flux, cfg.dtype = equation, flux, self.dtype_code
        cfg.sound_speed = sound_speed
        cfg.stream = self.stream.cuda_stream
        cfg.elems_per_block = elems_per_block
        cfg.device = device
        cfg.kernel = kernel
        cfg.mass = mass  # nat.NDG_MASS_LUMPED (the paper's) or nat.NDG_MASS_EXACT
        self.cfg = cfg
        self.dim, self.degree = dim, degree
        self.ctx = nat.ndg_create_ex(cfg)
        info = nat.ndg_info(self.ctx)
        self.nvar, self.npe, self.nelem = info.nvar, info.nodes_per_elem, info.nelem
        self.ndof, self.state_bytes = info.ndof, info.state_bytes
        self.kernel = info.kernel
        self.shape = (self.nvar, self.nelem, self.npe)

    # ---- state ----
    def set_state(self, U) -> None:
        if isinstance(U, torch.Tensor) and U.is_cuda:
            t = U.to(self.device, self.torch_dtype).contiguous()
            assert t.numel() == self.ndof
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            nat.ndg_set_state(self.ctx, t.data_ptr(), self.state_bytes, True)
            t.record_stream(self.stream)
        else:
            a = np.ascontiguousarray(U.cpu().numpy() if isinstance(U, torch.Tensor) else U, dtype=self.np_dtype)
            assert a.size == self.ndof
            nat.ndg_set_state(self.ctx, a.ctypes.data, self.state_bytes, False)

    def get_state(self, device: bool = False):
        """The state as a numpy array (host) or a CUDA tensor (device=True)."""
        if device:
            out = torch.empty(self.shape, dtype=self.torch_dtype, device=self.device)
            nat.ndg_get_state(self.ctx, out.data_ptr(), self.state_bytes, True)
            torch.cuda.current_stream(self.device).wait_stream(self.stream)
            return out
        out = np.empty(self.shape, dtype=self.np_dtype)
        nat.ndg_get_state(self.ctx, out.ctypes.data, self.state_bytes, False)
        return out

    # ---- stepping / diagnostics ----
    def step(self, dt: float, nsteps: int = 1, rk: int = nat.NDG_RK4) -> None:
        nat.ndg_step(self.ctx, dt, nsteps, rk)

    def norms(self, ref=None) -> dict:
        if ref is None:
            r = nat.ndg_norms(self.ctx, None, False, allow_nonfinite=True)
        else:
            a = np.ascontiguousarray(ref, dtype=self.np_dtype)
            r = nat.ndg_norms(self.ctx, a.ctypes.data, False, allow_nonfinite=True)
        return {"l2": r.l2, "linf": r.linf, "integral": np.array(r.integral[:self.nvar]),
                "max_speed": r.max_speed, "t": r.t, "steps": r.steps, "nonfinite": r.nonfinite}

    def stable_dt(self, cfl: float) -> float:
        return nat.ndg_stable_dt(self.ctx, cfl)

    def node_coords(self) -> np.ndarray:
        X = np.empty((self.dim, self.nelem, self.npe), dtype=np.float64)
        nat.ndg_node_coords(self.ctx, X.ctypes.data, X.size)
        return X

    def autotune(self, rk: int = nat.NDG_RK4):
        """(elements per block, ms per step) of the best tile; the mapping is in self.kernel."""
        best = nat.ndg_autotune(self.ctx, rk)
        self.kernel = nat.ndg_info(self.ctx).kernel
        return best

    def synchronize(self) -> None:
        nat.ndg_synchronize(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            nat.ndg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several solvers stepped together: one graph replay per RK step (ndg_batch_*)."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.handle = nat.ndg_batch_create([s.ctx for s in self.solvers])

    def step(self, dts, nsteps: int, rk: int = nat.NDG_RK4) -> None:
        nat.ndg_batch_step(self.handle, list(dts), nsteps, rk)

    def close(self) -> None:
        if self.handle:
            nat.ndg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
