"""GB300-native fundamental-scheme implicit FDTD (arXiv 2011.14043).

Python face of the C ABI in ``include/fdtd.h``.  Every step of the time
stepper runs in the CUDA library (``csrc/``); this module only marshals
arguments.  PyTorch is used for device buffers and the current CUDA stream.

    sim = Simulation(nx, ny, nz, dx, dy, dz, scheme="fadi", precision="f32", cfl=4.0)
    sim.set_field("ez", ez0)          # numpy (host) or torch CUDA tensor (device)
    sim.step(1000)
    ez = sim.get_field("ez")          # numpy; device=True gives a torch tensor
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import COMPS, PRECISIONS, SCHEMES, FdtdDesc, FdtdError, FdtdStats, check, lib

__all__ = ["Simulation", "Batch", "FdtdError", "comp_shape", "build", "energy_noalloc", "probe_fp64_fma"]


def comp_shape(comp: str, nx: int, ny: int, nz: int) -> tuple:
    return {
        "ex": (nz + 1, ny + 1, nx), "ey": (nz + 1, ny, nx + 1), "ez": (nz, ny + 1, nx + 1),
        "hx": (nz, ny, nx + 1), "hy": (nz, ny + 1, nx), "hz": (nz + 1, ny, nx),
    }[comp]


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _b
    return _b(force=force, verbose=verbose)


def _torch():
    import torch
    return torch


def probe_fp64_fma(iters: int = 20000) -> float:
    """Measured FP64 FMA throughput of the current device in FLOP/s (an FMA
    counts 2): the ALU roofline of the FP64 line solve."""
    v = ctypes.c_double()
    check(lib().fdtd_probe_fp64_fma(int(iters), ctypes.byref(v), None), "fdtd_probe_fp64_fma")
    return v.value


def energy_noalloc(fields: dict, nx, ny, nz, dx, dy, dz, eps_r=1.0, mu_r=1.0, out=None, stream=None):
    """Field energy of six CUDA tensors (compact Yee shapes) through
    ``fdtd_energy_noalloc``, which allocates no device memory: for callers
    that cannot allocate where they need the number.  ``out`` is a contiguous
    float64 CUDA tensor of at least one element on the fields' device
    (allocated here if omitted, by the caller's side); the result is written
    to its first element asynchronously on ``stream`` (default: the current
    stream of the fields' device).  Every argument is checked before anything
    is launched: tensors on different devices, or an ``out`` of another dtype
    or on the host, raise ValueError."""
    torch = _torch()
    if out is not None:
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or not out.is_cuda \
                or not out.is_contiguous() or out.numel() < 1:
            raise ValueError("out: need a contiguous float64 CUDA tensor with at least one element")
    ts = [fields[c] for c in COMPS]
    if not all(isinstance(t, torch.Tensor) for t in ts):
        raise ValueError("fields must be torch tensors")
    if len({t.dtype for t in ts}) != 1 or ts[0].dtype not in (torch.float32, torch.float64):
        raise ValueError("fields must share one dtype, float32 or float64")
    for c, t in zip(COMPS, ts):
        if not (t.is_cuda and t.is_contiguous()) or tuple(t.shape) != comp_shape(c, nx, ny, nz):
            raise ValueError(f"{c}: need a contiguous CUDA tensor of shape {comp_shape(c, nx, ny, nz)}")
    dev = ts[0].device
    if any(t.device != dev for t in ts) or (out is not None and out.device != dev):
        raise ValueError("the six fields and out must be on one CUDA device")
    prec = PRECISIONS["f64" if ts[0].dtype == torch.float64 else "f32"]
    with torch.cuda.device(dev):
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        ptrs = (ctypes.c_void_p * 6)(*[t.data_ptr() for t in ts])
        check(lib().fdtd_energy_noalloc(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                        float(eps_r), float(mu_r), prec, ptrs,
                                        ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                        ctypes.c_void_p(int(stream))), "fdtd_energy_noalloc")
    return out


class Simulation:
    """One grid on one GPU, bound to a CUDA stream (default: torch's current)."""

    def __init__(self, nx, ny, nz, dx, dy=None, dz=None, *, scheme="fadi", precision="f32",
                 dt=0.0, cfl=0.0, stream=None, tune=(0, 0)):
        dy = dx if dy is None else dy
        dz = dx if dz is None else dz
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.scheme = scheme
        self.precision = precision
        self.dtype = np.float64 if precision == "f64" else np.float32
        d = FdtdDesc()
        d.nx, d.ny, d.nz = self.nx, self.ny, self.nz
        d.dx, d.dy, d.dz = float(dx), float(dy), float(dz)
        d.dt = float(dt)
        d.cfl = float(cfl)
        d.scheme = SCHEMES[scheme]
        d.precision = PRECISIONS[precision]
        d.tune[0], d.tune[1] = int(tune[0]), int(tune[1])
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        self._stream = ctypes.c_void_p(int(stream))
        h = ctypes.c_void_p()
        check(lib().fdtd_create(ctypes.byref(d), self._stream, ctypes.byref(h)), "fdtd_create")
        self._h = h

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fdtd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- properties ----------------------------------------------------------
    @property
    def dt(self) -> float:
        v = ctypes.c_double()
        check(lib().fdtd_get_dt(self._h, ctypes.byref(v)), "fdtd_get_dt")
        return v.value

    @property
    def steps_done(self) -> int:
        v = ctypes.c_int64()
        check(lib().fdtd_steps_done(self._h, ctypes.byref(v)), "fdtd_steps_done")
        return v.value

    def shape(self, comp: str) -> tuple:
        return comp_shape(comp, self.nx, self.ny, self.nz)

    # -- problem set-up ------------------------------------------------------
    def set_material(self, eps_r_cell=None, mu_r_cell=None, sigma_cell=None):
        """Per-cell eps_r, mu_r and electric conductivity sigma [S/m]
        (shape (nz, ny, nx); None = 1, 1, 0)."""
        def ptr(a):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.shape != (self.nz, self.ny, self.nx):
                raise ValueError(f"material shape {a.shape} != {(self.nz, self.ny, self.nx)}")
            return a, a.ctypes.data_as(ctypes.c_void_p)
        ea, ep = ptr(eps_r_cell)
        ma, mp = ptr(mu_r_cell)
        if sigma_cell is None:
            check(lib().fdtd_set_material(self._h, ep, mp), "fdtd_set_material")
        else:
            sa, sp = ptr(sigma_cell)
            check(lib().fdtd_set_media(self._h, ep, mp, sp), "fdtd_set_media")

    def set_order(self, order: int):
        """Spatial difference order: 2 (Yee) or 4 (fourth-order staggered,
        PEC images); before the first step, uniform lossless media."""
        check(lib().fdtd_set_order(self._h, int(order)), "fdtd_set_order")

    def _put(self, fn, comp, data, what):
        c = COMPS[comp]
        if hasattr(data, "is_cuda") and data.is_cuda:
            torch = _torch()
            want = torch.float64 if self.precision == "f64" else torch.float32
            t = data.to(want).contiguous()
            if tuple(t.shape) != self.shape(comp):
                raise ValueError(f"{comp} shape {tuple(t.shape)} != {self.shape(comp)}")
            check(fn(self._h, c, ctypes.c_void_p(t.data_ptr()), 1), what)
            torch.cuda.current_stream().synchronize()
        else:
            a = np.ascontiguousarray(data, dtype=self.dtype)
            if a.shape != self.shape(comp):
                raise ValueError(f"{comp} shape {a.shape} != {self.shape(comp)}")
            check(fn(self._h, c, a.ctypes.data_as(ctypes.c_void_p), 0), what)

    def _get(self, fn, comp, device, what, out=None):
        c = COMPS[comp]
        if out is not None:
            if out.shape != self.shape(comp) or out.dtype != self.dtype or not out.flags.c_contiguous:
                raise ValueError(f"out must be a C-contiguous {self.dtype.__name__} array of shape {self.shape(comp)}")
            check(fn(self._h, c, out.ctypes.data_as(ctypes.c_void_p), 0), what)
            return out
        if device:
            torch = _torch()
            t = torch.empty(self.shape(comp), dtype=torch.float64 if self.precision == "f64" else torch.float32,
                            device="cuda")
            check(fn(self._h, c, ctypes.c_void_p(t.data_ptr()), 1), what)
            return t
        a = np.empty(self.shape(comp), dtype=self.dtype)
        check(fn(self._h, c, a.ctypes.data_as(ctypes.c_void_p), 0), what)
        return a

    def set_field(self, comp: str, data):
        self._put(lib().fdtd_set_field, comp, data, "fdtd_set_field")

    def set_fields(self, fields: dict):
        for c, v in fields.items():
            self.set_field(c, v)

    def get_field(self, comp: str, device: bool = False, out=None):
        """Physical field component; ``out`` (host array, e.g. pinned) is filled in place."""
        return self._get(lib().fdtd_get_field, comp, device, "fdtd_get_field", out)

    def get_fields(self, device: bool = False) -> dict:
        return {c: self.get_field(c, device) for c in COMPS}

    def set_state(self, comp: str, data):
        self._put(lib().fdtd_set_state, comp, data, "fdtd_set_state")

    def get_state(self, comp: str, device: bool = False):
        return self._get(lib().fdtd_get_state, comp, device, "fdtd_get_state")

    def set_source(self, comp: str, i: int, j: int, k: int, current):
        cur = np.ascontiguousarray(current, dtype=np.float64)
        check(lib().fdtd_set_source(self._h, COMPS[comp], int(i), int(j), int(k),
                                    cur.ctypes.data_as(ctypes.c_void_p), cur.size), "fdtd_set_source")
        self._src_keep = cur

    def add_probe(self, comp: str, i: int, j: int, k: int) -> int:
        pid = ctypes.c_int()
        check(lib().fdtd_add_probe(self._h, COMPS[comp], int(i), int(j), int(k), ctypes.byref(pid)),
              "fdtd_add_probe")
        return pid.value

    def get_probe(self, pid: int, n: int) -> np.ndarray:
        out = np.empty(int(n), dtype=np.float64)
        check(lib().fdtd_get_probe(self._h, int(pid), out.ctypes.data_as(ctypes.c_void_p), int(n)),
              "fdtd_get_probe")
        return out

    # -- stepping and reductions -----------------------------------------------
    def step(self, n: int = 1):
        check(lib().fdtd_step(self._h, int(n)), "fdtd_step")

    def synchronize(self):
        check(lib().fdtd_synchronize(self._h), "fdtd_synchronize")

    def set_timing(self, enable: bool):
        check(lib().fdtd_set_timing(self._h, 1 if enable else 0), "fdtd_set_timing")

    def stats(self) -> dict:
        st = FdtdStats()
        check(lib().fdtd_get_stats(self._h, ctypes.byref(st)), "fdtd_get_stats")
        return {"launches": st.launches, "timed_launches": list(st.timed_launches),
                "timed_ms": list(st.timed_ms), "bytes_per_launch": list(st.bytes_per_launch)}

    def reset_stats(self):
        check(lib().fdtd_reset_stats(self._h), "fdtd_reset_stats")

    def energy(self) -> tuple:
        out = (ctypes.c_double * 2)()
        check(lib().fdtd_energy(self._h, out), "fdtd_energy")
        return out[0], out[1]


class Batch:
    """Many independent grids stepped together (launch groups per line
    direction and procedure, or one persistent launch per procedure, for the
    whole batch; one CUDA graph per batch step).  The
    Simulation objects stay usable for set/get/energy and must share scheme,
    precision and stream; they must outlive the batch."""

    def __init__(self, sims):
        self.sims = list(sims)
        if not self.sims:
            raise ValueError("empty batch")
        arr = (ctypes.c_void_p * len(self.sims))(*[s_._h.value for s_ in self.sims])
        h = ctypes.c_void_p()
        check(lib().fdtd_batch_create(arr, len(self.sims), self.sims[0]._stream, ctypes.byref(h)),
              "fdtd_batch_create")
        self._h = h

    def step(self, n: int = 1):
        check(lib().fdtd_batch_step(self._h, int(n)), "fdtd_batch_step")

    def config(self) -> dict:
        """Launch shape in use (tuned on the first step unless fixed) and the
        tuned per-direction times of one step's launches (ms)."""
        cfg = (ctypes.c_int32 * 6)()
        ms = (ctypes.c_double * 3)()
        check(lib().fdtd_batch_get_config(self._h, cfg, ms), "fdtd_batch_get_config")
        return {"y": (cfg[0], cfg[1]), "z": (cfg[2], cfg[3]), "x_warps_per_block": cfg[4], "x_pack": cfg[5],
                "tuned_ms": {"y": ms[0], "z": ms[1], "x": ms[2]}}

    def set_config(self, y=None, z=None, x_warps_per_block=8, x_pack=1):
        """Fix the launch shape: y, z = (lanes, L); x_pack 1 lets short x lines of
        grids with per-node media share warps; None for y and z returns to tuning."""
        if y is None and z is None:
            check(lib().fdtd_batch_set_config(self._h, None), "fdtd_batch_set_config")
            return
        cfg = (ctypes.c_int32 * 6)(y[0], y[1], z[0], z[1], x_warps_per_block, x_pack)
        check(lib().fdtd_batch_set_config(self._h, cfg), "fdtd_batch_set_config")

    def launches_per_step(self) -> int:
        v = ctypes.c_int64()
        check(lib().fdtd_batch_launches(self._h, ctypes.byref(v)), "fdtd_batch_launches")
        return v.value

    _MODES = {"auto": -1, "launches": 0, "persistent": 1}

    def set_mode(self, mode: str = "auto"):
        """How a step runs: "launches" (a graph of shape-uniform launches),
        "persistent" (one persistent launch per procedure over a work list
        of every grid's lines), or "auto" (the faster, timed at the first
        step)."""
        check(lib().fdtd_batch_set_mode(self._h, self._MODES[mode]), "fdtd_batch_set_mode")

    def mode(self) -> dict:
        """The mode in use (after a step) and the tuned time of one step in
        each mode (ms; 0 when not timed)."""
        v = ctypes.c_int32()
        ms = (ctypes.c_double * 2)()
        check(lib().fdtd_batch_get_mode(self._h, ctypes.byref(v), ms), "fdtd_batch_get_mode")
        return {"mode": "persistent" if v.value else "launches",
                "tuned_step_ms": {"launches": ms[0], "persistent": ms[1]}}

    def synchronize(self):
        self.sims[0].synchronize()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fdtd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
