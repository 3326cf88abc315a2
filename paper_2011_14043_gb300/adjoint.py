"""Differentiable FADI: the probe energy of a cavity run as a function of the
per-cell relative permittivity, with its gradient from the library's
hand-written discrete adjoint (``fdtd_adj_*`` in include/fdtd.h) behind a
``torch.autograd.Function``.

    prob = ProbeEnergyProblem(192, 192, 192, 1e-3, cfl=4.0, steps=500,
                              checkpoint_every=25, probe_block=(140, 144, 94, 98, 94, 98),
                              source=("ez", 48, 96, 96, current))
    eps = torch.ones(192, 192, 192, dtype=torch.float64, requires_grad=True)
    J = prob.objective(eps)      # forward run on the GPU
    J.backward()                 # adjoint run on the GPU; eps.grad = dJ/d eps_r

J = sum over steps n = 1..steps and over the probe E samples of (E^n)^2,
with E^n the FADI output field after step n.  Only argument marshalling
happens here: the forward steps, the checkpointing, the recomputation and
the adjoint procedures all run in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Simulation
from ._lib import check, lib

__all__ = ["ProbeEnergyProblem", "AdjointRun"]


class AdjointRun:
    """One forward run with its adjoint context (owns both handles)."""

    def __init__(self, prob: "ProbeEnergyProblem", eps_r_cell: np.ndarray):
        p = prob
        self.sim = Simulation(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, scheme="fadi", precision=p.precision,
                              dt=p.dt, cfl=p.cfl, stream=p.stream, tune=(0, 2))
        self.sim.set_material(eps_r_cell)
        if p.fields is not None:
            self.sim.set_fields(p.fields)
        if p.source is not None:
            self.sim.set_source(*p.source)
        blk = (ctypes.c_int32 * 6)(*[int(v) for v in p.probe_block])
        h = ctypes.c_void_p()
        check(lib().fdtd_adj_create(self.sim._h, blk, int(p.steps), int(p.checkpoint_every), ctypes.byref(h)),
              "fdtd_adj_create")
        self._h = h

    def memory_bytes(self) -> int:
        v = ctypes.c_int64()
        check(lib().fdtd_adj_memory(self._h, ctypes.byref(v)), "fdtd_adj_memory")
        return v.value

    def forward(self) -> float:
        J = ctypes.c_double()
        check(lib().fdtd_adj_forward(self._h, ctypes.byref(J)), "fdtd_adj_forward")
        return J.value

    def backward(self, jbar: float = 1.0, out=None):
        """jbar * dJ/d eps_r per cell: a float64 CUDA tensor of shape (nz, ny, nx)
        (``out`` if given), or a numpy array when ``out`` is a numpy array."""
        s = self.sim
        if isinstance(out, np.ndarray):
            if out.shape != (s.nz, s.ny, s.nx) or out.dtype != np.float64 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array of shape (nz, ny, nx)")
            check(lib().fdtd_adj_backward(self._h, float(jbar), out.ctypes.data_as(ctypes.c_void_p), 0),
                  "fdtd_adj_backward")
            return out
        import torch
        if out is None:
            out = torch.empty((s.nz, s.ny, s.nx), dtype=torch.float64, device="cuda")
        if not (out.is_cuda and out.is_contiguous() and out.dtype == torch.float64):
            raise ValueError("out must be a contiguous float64 CUDA tensor")
        check(lib().fdtd_adj_backward(self._h, float(jbar), ctypes.c_void_p(out.data_ptr()), 1),
              "fdtd_adj_backward")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fdtd_adj_destroy(self._h)
            self._h = ctypes.c_void_p()
        if getattr(self, "sim", None) is not None:
            self.sim.close()
            self.sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProbeEnergyProblem:
    """A FADI run (grid, time step, source, initial field, probe block, step
    count, checkpoint spacing) whose probe energy is differentiated with
    respect to eps_r of every cell."""

    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, *, steps, probe_block, dt=0.0, cfl=0.0,
                 precision="f32", checkpoint_every=25, source=None, fields=None, stream=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx = float(dx)
        self.dy = float(dx if dy is None else dy)
        self.dz = float(dx if dz is None else dz)
        self.steps = int(steps)
        self.probe_block = tuple(int(v) for v in probe_block)
        self.dt, self.cfl = float(dt), float(cfl)
        self.precision = precision
        self.checkpoint_every = int(checkpoint_every)
        self.source = source
        self.fields = fields
        self.stream = stream

    def _eps_host(self, eps_r) -> np.ndarray:
        if hasattr(eps_r, "detach"):
            eps_r = eps_r.detach().to("cpu").numpy()
        a = np.ascontiguousarray(eps_r, dtype=np.float64)
        if a.shape != (self.nz, self.ny, self.nx):
            raise ValueError(f"eps_r shape {a.shape} != {(self.nz, self.ny, self.nx)}")
        return a

    def run(self, eps_r) -> AdjointRun:
        """Forward run; the returned object holds J (``.J``) and can run the adjoint."""
        r = AdjointRun(self, self._eps_host(eps_r))
        r.J = r.forward()
        return r

    def value(self, eps_r) -> float:
        """J alone (no adjoint kept)."""
        r = self.run(eps_r)
        J = r.J
        r.close()
        return J

    def objective(self, eps_r):
        """Differentiable J(eps_r) (a float64 scalar tensor on eps_r's device)."""
        return _ProbeEnergy.apply(eps_r, self)


def _make_function():
    import torch

    class ProbeEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, eps_r, prob):
            run = prob.run(eps_r)
            ctx.run = run
            ctx.meta = (eps_r.dtype, eps_r.device)
            return torch.tensor(run.J, dtype=torch.float64, device=eps_r.device)

        @staticmethod
        def backward(ctx, gJ):
            run = ctx.run
            g = run.backward(float(gJ))
            run.close()
            ctx.run = None
            dtype, device = ctx.meta
            return g.to(device=device, dtype=dtype), None

    return ProbeEnergy


class _Lazy:
    fn = None

    @classmethod
    def apply(cls, *a):
        if cls.fn is None:
            cls.fn = _make_function()
        return cls.fn.apply(*a)


_ProbeEnergy = _Lazy
