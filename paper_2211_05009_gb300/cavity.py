"""Object wrapper over the C ABI: one lid-driven cavity on the GPU.

PyTorch provides the device buffers the outputs land in and the CUDA stream the library queues
on; every number is computed by the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Cavity:
    """A D2Q9 lid-driven cavity of nx x ny nodes (walls included) on cuda:0.

    Either ``Re`` (tau from Re = U nx / nu, nu = (tau - 1/2)/3) or ``tau`` must be given.
    ``dtype`` is the population storage: f64, f32, f32s, f16s, bf16s or q16s.
    """

    def __init__(self, nx: int, ny: int, Re: float | None = None, U: float = 0.1, dtype: str = "f32s",
                 tau: float | None = None, corners_moving: bool = False, stream: torch.cuda.Stream | None = None):
        if (Re is None) == (tau is None):
            raise ValueError("give exactly one of Re and tau")
        flags = B.LBM_FLAG_LID_CORNERS_MOVING if corners_moving else 0
        if Re is not None:
            self.ctx = B.lbm_create_flags(nx, ny, Re, U, dtype, flags)
        else:
            self.ctx = B.lbm_create_ex(nx, ny, tau, U, dtype, flags)
        self.nx, self.ny, self.dtype = nx, ny, dtype
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        B.lbm_set_stream(self.ctx, self.stream.cuda_stream)
        self._probes = []

    # lifetime
    def close(self):
        if getattr(self, "ctx", None):
            B.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def info(self) -> B.lbm_info:
        return B.lbm_get_info(self.ctx)

    @property
    def tau(self) -> float:
        return self.info.tau

    @property
    def step_count(self) -> int:
        return self.info.step

    # time stepping
    def step(self, n: int = 1):
        B.lbm_step(self.ctx, n)
        return self

    def run_to_residual(self, tol: float, max_steps: int):
        """(converged, steps taken)."""
        rc, done = B.lbm_run_to_residual(self.ctx, tol, max_steps)
        return rc == B.LBM_OK, done

    # observables (torch CUDA tensors unless host=True)
    def _empty(self, shape, host: bool):
        if host:
            return np.empty(shape, dtype=np.float64)
        return torch.empty(shape, dtype=torch.float64, device="cuda")

    def moments(self, host: bool = False):
        rho, ux, uy = (self._empty((self.ny, self.nx), host) for _ in range(3))
        B.lbm_moments(self.ctx, rho, ux, uy)
        return rho, ux, uy

    def populations(self, host: bool = False):
        f = self._empty((9, self.ny, self.nx), host)
        B.lbm_get_populations(self.ctx, f)
        return f

    def set_populations(self, f):
        B.lbm_set_populations(self.ctx, f)

    def set_moments(self, rho, ux, uy, neq: bool = False):
        B.lbm_set_moments(self.ctx, rho, ux, uy, B.LBM_INIT_NEQ if neq else 0)

    def residual(self) -> float:
        return B.lbm_residual(self.ctx)

    def mass(self) -> float:
        return B.lbm_mass(self.ctx)

    def stream_function(self, psi: bool = False, host: bool = False):
        """(psi_min, xc, yc[, psi field])."""
        buf = self._empty((self.ny, self.nx), host) if psi else None
        vmin, xc, yc = B.lbm_stream_function(self.ctx, buf)
        return (vmin, xc, yc, buf) if psi else (vmin, xc, yc)

    def stream_function_window(self, i0, i1, j0, j1):
        return B.lbm_stream_function_window(self.ctx, i0, i1, j0, j1)

    def probe(self, x: float, y: float, every: int = 2, cap: int = 1 << 16):
        """Add an observing point; returns (index, device series tensor [cap, 2])."""
        series = torch.zeros((cap, 2), dtype=torch.float64, device="cuda")
        q = B.lbm_probe(self.ctx, x, y, every, series, cap)
        self._probes.append(series)
        return q, series

    def probe_count(self, q: int) -> int:
        return B.lbm_probe_count(self.ctx, q)

    def save(self, path: str):
        B.lbm_save(self.ctx, path)

    def load(self, path: str):
        B.lbm_load(self.ctx, path)
