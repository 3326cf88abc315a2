"""Seeded synthetic inputs for the implicit FDTD workloads.

This module is shared by the CPU oracle and by the CUDA path's tests and
benchmark.  It only *creates inputs* (initial fields, per-cell materials,
source currents, grid sizes); it holds none of the time-stepping arithmetic.

Array layout everywhere: C-contiguous ``[k, j, i]`` (x fastest).  Yee sample
positions (cell indices i, j, k; spacing dx, dy, dz):

    Ex (i+1/2, j, k)      shape (nz+1, ny+1, nx)
    Ey (i, j+1/2, k)      shape (nz+1, ny, nx+1)
    Ez (i, j, k+1/2)      shape (nz, ny+1, nx+1)
    Hx (i, j+1/2, k+1/2)  shape (nz, ny, nx+1)
    Hy (i+1/2, j, k+1/2)  shape (nz, ny+1, nx)
    Hz (i+1/2, j+1/2, k)  shape (nz+1, ny, nx)

The paper (Sec. III) only says "second-order central differencing on Yee
cells"; the standard Yee staggering above is the reading used throughout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")


def comp_shape(comp: str, nx: int, ny: int, nz: int) -> tuple:
    """Shape ``(kz, jy, ix)`` of one Yee component on an nx*ny*nz cell grid."""
    return {
        "ex": (nz + 1, ny + 1, nx),
        "ey": (nz + 1, ny, nx + 1),
        "ez": (nz, ny + 1, nx + 1),
        "hx": (nz, ny, nx + 1),
        "hy": (nz, ny + 1, nx),
        "hz": (nz + 1, ny, nx),
    }[comp]


def comp_offsets(comp: str) -> tuple:
    """Half-cell offsets (ox, oy, oz) of a component's samples (Yee)."""
    return {
        "ex": (0.5, 0.0, 0.0),
        "ey": (0.0, 0.5, 0.0),
        "ez": (0.0, 0.0, 0.5),
        "hx": (0.0, 0.5, 0.5),
        "hy": (0.5, 0.0, 0.5),
        "hz": (0.5, 0.5, 0.0),
    }[comp]


def zero_fields(nx: int, ny: int, nz: int, dtype=np.float64) -> dict:
    return {c: np.zeros(comp_shape(c, nx, ny, nz), dtype=dtype) for c in COMPONENTS}


# ---------------------------------------------------------------------------
# 2-D (nz = 1) Gaussian Ez pulse
# ---------------------------------------------------------------------------

def gaussian_ez_2d(nx: int, ny: int, sigma_cells: float, seed: int) -> dict:
    """Initial fields: Ez = exp(-((i-ic)^2+(j-jc)^2)/(2 sigma^2)) on the Ez
    nodes of a 2-D grid run as nz = 1; (ic, jc) are integers drawn uniformly
    from {n//5 .. n - n//5} per axis ({12..52} on a 64 x 64 grid); wall nodes
    zeroed; all else 0."""
    rng = np.random.default_rng(seed)
    ic = int(rng.integers(nx // 5, nx - nx // 5 + 1))
    jc = int(rng.integers(ny // 5, ny - ny // 5 + 1))
    f = zero_fields(nx, ny, 1)
    j, i = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ez = np.exp(-((i - ic) ** 2 + (j - jc) ** 2) / (2.0 * sigma_cells ** 2))
    ez[0, :] = 0.0
    ez[-1, :] = 0.0
    ez[:, 0] = 0.0
    ez[:, -1] = 0.0
    f["ez"][0] = ez
    return f, (ic, jc)


# ---------------------------------------------------------------------------
# PEC cavity eigenmode superpositions (workloads 2 and 4)
# ---------------------------------------------------------------------------

@dataclass
class Mode:
    m: int
    n: int
    p: int
    amp: float
    pol: tuple  # unit polarisation (ax, ay, az)


def random_modes(seed_or_rng, nx, ny, nz, dx, dy, dz, count=8, mmax=16):
    """Draw ``count`` distinct cavity modes (m, n, p) uniform in
    {1..mmax}^3 (capped at the cell counts minus one), N(0,1) amplitudes and a
    random unit polarisation orthogonal to the Yee wave vector
    k'_xi = (2/d_xi) sin(k_xi d_xi / 2), which makes the sampled field
    divergence-free on the grid."""
    rng = seed_or_rng if isinstance(seed_or_rng, np.random.Generator) else np.random.default_rng(seed_or_rng)
    caps = (min(mmax, nx - 1), min(mmax, ny - 1), min(mmax, nz - 1))
    seen = set()
    modes = []
    while len(modes) < count:
        mnp = tuple(int(rng.integers(1, c + 1)) for c in caps)
        if mnp in seen:
            continue
        seen.add(mnp)
        amp = float(rng.standard_normal())
        kp = np.array([
            (2.0 / dx) * math.sin(mnp[0] * math.pi / nx / 2.0),
            (2.0 / dy) * math.sin(mnp[1] * math.pi / ny / 2.0),
            (2.0 / dz) * math.sin(mnp[2] * math.pi / nz / 2.0),
        ])
        khat = kp / np.linalg.norm(kp)
        while True:
            g = rng.standard_normal(3)
            a = g - khat * np.dot(g, khat)
            na = np.linalg.norm(a)
            if na > 1e-6:
                break
        modes.append(Mode(mnp[0], mnp[1], mnp[2], amp, tuple(a / na)))
    return modes


def mode_e_shape(mode: Mode, nx, ny, nz, unit_amp: bool = False) -> dict:
    """E field of one PEC cavity mode sampled on the Yee E positions:
    Ex ~ ax cos(kx x) sin(ky y) sin(kz z), Ey ~ ay sin cos sin,
    Ez ~ az sin sin cos, with k_xi = m_xi pi / N_xi (positions in cells)."""
    kx = mode.m * math.pi / nx
    ky = mode.n * math.pi / ny
    kz = mode.p * math.pi / nz
    amp = 1.0 if unit_amp else mode.amp
    out = {}
    for c, trig in (("ex", (np.cos, np.sin, np.sin)),
                    ("ey", (np.sin, np.cos, np.sin)),
                    ("ez", (np.sin, np.sin, np.cos))):
        sh = comp_shape(c, nx, ny, nz)
        ox, oy, oz = comp_offsets(c)
        x = (np.arange(sh[2]) + ox) * kx
        y = (np.arange(sh[1]) + oy) * ky
        z = (np.arange(sh[0]) + oz) * kz
        a = mode.pol["xyz".index(c[1])]
        out[c] = amp * a * (trig[2](z)[:, None, None] * trig[1](y)[None, :, None] * trig[0](x)[None, None, :])
    return out


def mode_sum_fields(modes, nx, ny, nz) -> dict:
    f = zero_fields(nx, ny, nz)
    for md in modes:
        sh = mode_e_shape(md, nx, ny, nz)
        for c in ("ex", "ey", "ez"):
            f[c] += sh[c]
    # PEC: tangential E exactly zero on the walls (the sines vanish up to rounding)
    f["ex"][:, 0, :] = 0; f["ex"][:, -1, :] = 0; f["ex"][0] = 0; f["ex"][-1] = 0
    f["ey"][:, :, 0] = 0; f["ey"][:, :, -1] = 0; f["ey"][0] = 0; f["ey"][-1] = 0
    f["ez"][:, :, 0] = 0; f["ez"][:, :, -1] = 0; f["ez"][:, 0, :] = 0; f["ez"][:, -1, :] = 0
    return f


# ---------------------------------------------------------------------------
# Per-cell permittivity blocks (workloads 3 and 4)
# ---------------------------------------------------------------------------

def eps_blocks(seed_or_rng, nx, ny, nz, lo, hi, count=16):
    """Per-cell eps_r (shape (nz, ny, nx)): background 1, then ``count``
    axis-aligned blocks, per-axis size uniform in {N/16..N/4} (at least 1),
    corner uniform in {0..N-size}, value uniform in [lo, hi]; later blocks
    overwrite earlier ones."""
    rng = seed_or_rng if isinstance(seed_or_rng, np.random.Generator) else np.random.default_rng(seed_or_rng)
    eps = np.ones((nz, ny, nx))
    dims = (nx, ny, nz)
    for _ in range(count):
        lo_hi = []
        for n in dims:
            smin = max(1, n // 16)
            smax = max(smin, n // 4)
            s = int(rng.integers(smin, smax + 1))
            c0 = int(rng.integers(0, n - s + 1))
            lo_hi.append((c0, c0 + s))
        val = float(rng.uniform(lo, hi))
        (x0, x1), (y0, y1), (z0, z1) = lo_hi
        eps[z0:z1, y0:y1, x0:x1] = val
    return eps


# ---------------------------------------------------------------------------
# Source current
# ---------------------------------------------------------------------------

def gaussian_pulse_params(f0: float, frac_bw: float):
    """Modulated-Gaussian parameters: the -3 dB power full width of the
    spectrum is frac_bw*f0, so sigma_f = (frac_bw f0 / 2)/sqrt(ln 2),
    sigma_t = 1/(2 pi sigma_f), delay t0 = 5 sigma_t."""
    sigma_f = 0.5 * frac_bw * f0 / math.sqrt(math.log(2.0))
    sigma_t = 1.0 / (2.0 * math.pi * sigma_f)
    return sigma_t, 5.0 * sigma_t


def dipole_current(t, f0: float = 10e9, frac_bw: float = 0.5):
    """Dipole current I(t) = exp(-(t-t0)^2/(2 sigma_t^2)) sin(2 pi f0 (t-t0)) [A]."""
    sigma_t, t0 = gaussian_pulse_params(f0, frac_bw)
    t = np.asarray(t, dtype=np.float64)
    return np.exp(-((t - t0) ** 2) / (2.0 * sigma_t ** 2)) * np.sin(2.0 * math.pi * f0 * (t - t0))


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    cfl: float
    steps: int
    scheme: str
    fields: dict = field(default_factory=dict)
    eps_r: np.ndarray | None = None
    source: dict | None = None
    probes: list = field(default_factory=list)
    extra: dict = field(default_factory=dict)


def workload_2d_gaussian(seed: int = 1, n: int = 64, steps: int = 200) -> Workload:
    f, centre = gaussian_ez_2d(n, n, 6.0, seed)
    return Workload("2d_fadi_gaussian", n, n, 1, 1e-3, 1e-3, 1e-3, 5.0, steps, "fadi",
                    fields=f, probes=[("ez", 16, 16, 0)], extra={"centre": centre})


def workload_cavity_modes(seed: int = 2, n: int = 128, steps: int = 1000, cfl: float = 4.0,
                          nmodes: int = 8) -> Workload:
    d = 1e-3
    modes = random_modes(seed, n, n, n, d, d, d, count=nmodes)
    f = mode_sum_fields(modes, n, n, n)
    return Workload(f"cavity_modes_{n}", n, n, n, d, d, d, cfl, steps, "fadi",
                    fields=f, extra={"modes": modes})


def workload_dipole_blocks(seed: int = 3, n: int = 256, steps: int = 1000, cfl: float = 8.0,
                           scheme: str = "flod") -> Workload:
    d = 0.5e-3
    eps = eps_blocks(seed, n, n, n, 1.0, 10.0)
    c = n // 2
    return Workload(f"dipole_blocks_{n}", n, n, n, d, d, d, cfl, steps, scheme,
                    fields=zero_fields(n, n, n), eps_r=eps,
                    source={"comp": "ez", "i": c, "j": c, "k": c, "f0": 10e9, "frac_bw": 0.5})


def workload_batch(seed: int = 4, count: int = 64, steps: int = 500):
    """Many independent cavities: sizes nx in {32..160}, ny in {32..96},
    nz in {32..128}, CFL uniform in [2, 10], eps_r blocks uniform in [1, 4],
    8-mode initial field, cell size 1 mm."""
    rng = np.random.default_rng(seed)
    out = []
    d = 1e-3
    for b in range(count):
        nx = int(rng.integers(32, 161)); ny = int(rng.integers(32, 97)); nz = int(rng.integers(32, 129))
        cfl = float(rng.uniform(2.0, 10.0))
        eps = eps_blocks(rng, nx, ny, nz, 1.0, 4.0)
        modes = random_modes(rng, nx, ny, nz, d, d, d, count=8)
        out.append(Workload(f"batch_{b}", nx, ny, nz, d, d, d, cfl, steps, "fadi",
                            fields=mode_sum_fields(modes, nx, ny, nz), eps_r=eps,
                            extra={"modes": modes}))
    return out


def workload_adjoint(seed: int = 5, n: int = 192, steps: int = 500, cfl: float = 4.0, region=(64, 128),
                     checkpoint_every: int = 25) -> Workload:
    """Differentiable FADI run: eps_r uniform in [1, 6] per cell inside the
    central design cube [region)^3, 1 elsewhere; 1 mm cells; z-directed dipole
    (10 GHz, 50% bandwidth modulated Gaussian) at the Ez sample (48, 96, 96);
    objective = probe energy over the E samples of cells
    [140, 144) x [94, 98) x [94, 98) over all steps.  Sample positions scale
    with n / 192 for smaller test grids."""
    rng = np.random.default_rng(seed)
    d = 1e-3
    eps = np.ones((n, n, n))
    lo, hi = (region[0] * n) // 192, (region[1] * n) // 192
    eps[lo:hi, lo:hi, lo:hi] = rng.uniform(1.0, 6.0, (hi - lo,) * 3)
    s = lambda v: (v * n) // 192
    block = (s(140), s(140) + max(1, s(4)), s(94), s(94) + max(1, s(4)), s(94), s(94) + max(1, s(4)))
    return Workload(f"adjoint_{n}", n, n, n, d, d, d, cfl, steps, "fadi",
                    fields=zero_fields(n, n, n), eps_r=eps,
                    source={"comp": "ez", "i": s(48), "j": s(96), "k": s(96), "f0": 10e9, "frac_bw": 0.5},
                    extra={"probe_block": block, "checkpoint_every": checkpoint_every,
                           "region": (lo, hi)})
