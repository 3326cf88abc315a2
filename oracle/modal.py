"""Closed-form evolution of PEC-cavity modes (vacuum, any grid size).

On the Yee grid with PEC walls, the fields of one cavity mode (m, n, p),
k_xi = m_xi pi / L_xi, span a 6-dimensional space invariant under both
splitting operators A and B of Eqs. 33-34:

    Ex ~ cos(kx x) sin(ky y) sin(kz z)     Hx ~ sin(kx x) cos(ky y) cos(kz z)
    Ey ~ sin(kx x) cos(ky y) sin(kz z)     Hy ~ cos(kx x) sin(ky y) cos(kz z)
    Ez ~ sin(kx x) sin(ky y) cos(kz z)     Hz ~ cos(kx x) cos(ky y) sin(kz z)

each sampled at the component's own Yee positions.  A staggered first
difference maps sin to +kappa cos and cos to -kappa sin, with
kappa_xi = (2/d_xi) sin(k_xi d_xi / 2), so on this space A and B are 6 x 6
matrices.  Any of the splitting schemes of Sec. II then evolves the mode's
6 amplitudes by a 6 x 6 amplification matrix, and the field after n steps
is the sum over modes of amplitudes x shapes.  This gives the exact
(FP64) field of a multi-mode cavity run at any size and step count without
running the stepper: a full-size reference for the CUDA path, pinned
against the structured oracle on small grids.
"""
from __future__ import annotations

import math

import numpy as np

from .grid import EPS0, MU0, Grid

# component order of the 6-vectors
ORDER = ("ex", "ey", "ez", "hx", "hy", "hz")
# (x, y, z) trig of each component: "c" = cos, "s" = sin
TRIG = {"ex": "css", "ey": "scs", "ez": "ssc", "hx": "scc", "hy": "csc", "hz": "ccs"}
OFFSET = {"ex": (0.5, 0, 0), "ey": (0, 0.5, 0), "ez": (0, 0, 0.5),
          "hx": (0, 0.5, 0.5), "hy": (0.5, 0, 0.5), "hz": (0.5, 0.5, 0)}


def kappa(order: int, theta: float, d: float) -> float:
    """Symbol of the staggered first difference on sin/cos samples, theta =
    k d: (2/d) sin(theta/2) for the Yee difference; (2/d)(9/8 sin(theta/2) -
    1/24 sin(3 theta/2)) for the fourth-order one (with PEC images the cavity
    modes stay exact eigenfunctions)."""
    if order == 4:
        return (2.0 / d) * (9.0 / 8.0 * math.sin(theta / 2.0) - 1.0 / 24.0 * math.sin(1.5 * theta))
    return (2.0 / d) * math.sin(theta / 2.0)


def mode_operators(grid: Grid, m: int, n: int, p: int, eps: float = EPS0, mu: float = MU0,
                   sigma: float = 0.0):
    """A and B (Eqs. 33-34) restricted to the mode's 6-dimensional space; a
    homogeneous conductivity sigma puts -sigma/(2 eps) on the E diagonal of
    each (the split loss of oracle.grid)."""
    kx = kappa(grid.order, m * math.pi / grid.nx, grid.dx)
    ky = kappa(grid.order, n * math.pi / grid.ny, grid.dy)
    kz = kappa(grid.order, p * math.pi / grid.nz, grid.dz)
    EX, EY, EZ, HX, HY, HZ = range(6)
    A = np.zeros((6, 6))
    B = np.zeros((6, 6))
    # A: +(1/eps) d_y Hz, +(1/eps) d_z Hx, +(1/eps) d_x Hy; +(1/mu) d_z Ey, +(1/mu) d_x Ez, +(1/mu) d_y Ex
    A[EX, HZ] = -ky / eps   # d_y of cos -> -kappa sin
    A[EY, HX] = -kz / eps
    A[EZ, HY] = -kx / eps
    A[HX, EY] = +kz / mu    # d_z of sin -> +kappa cos
    A[HY, EZ] = +kx / mu
    A[HZ, EX] = +ky / mu
    # B: -(1/eps) d_z Hy, -(1/eps) d_x Hz, -(1/eps) d_y Hx; -(1/mu) d_y Ez, -(1/mu) d_z Ex, -(1/mu) d_x Ey
    B[EX, HY] = +kz / eps
    B[EY, HZ] = +kx / eps
    B[EZ, HX] = +ky / eps
    B[HX, EZ] = -ky / mu
    B[HY, EX] = -kz / mu
    B[HZ, EY] = -kx / mu
    for q in (EX, EY, EZ):
        A[q, q] = B[q, q] = -0.5 * sigma / eps
    return A, B


def amplification(scheme: str, dt: float, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """One time step of a splitting scheme on a mode (original forms of Sec. II;
    the fundamental forms give the same fields)."""
    I = np.eye(6)

    def cn(O, tau):
        return np.linalg.solve(I - tau * O, I + tau * O)

    if scheme in ("adi", "fadi"):        # Eq. 1
        t = dt / 2
        return np.linalg.solve(I - t * B, I + t * A) @ np.linalg.solve(I - t * A, I + t * B)
    if scheme in ("lod1", "flod"):       # Eq. 11
        return cn(B, dt / 2) @ cn(A, dt / 2)
    if scheme in ("ss2", "fss"):         # Eq. 16
        return cn(A, dt / 4) @ cn(B, dt / 2) @ cn(A, dt / 4)
    raise ValueError(scheme)


def mode_shape(grid: Grid, comp: str, m: int, n: int, p: int) -> np.ndarray:
    """Unit-amplitude shape of one component of mode (m, n, p) on its Yee samples."""
    from .grid import shape as comp_shape
    sh = comp_shape(comp, grid.nx, grid.ny, grid.nz)
    ox, oy, oz = OFFSET[comp]
    fx, fy, fz = (np.cos if t == "c" else np.sin for t in TRIG[comp])
    x = fx((np.arange(sh[2]) + ox) * (m * math.pi / grid.nx))
    y = fy((np.arange(sh[1]) + oy) * (n * math.pi / grid.ny))
    z = fz((np.arange(sh[0]) + oz) * (p * math.pi / grid.nz))
    return z[:, None, None] * y[None, :, None] * x[None, None, :]


def evolve_modes(grid: Grid, dt: float, scheme: str, modes, steps: int, eps: float = EPS0,
                 sigma: float = 0.0):
    """6-vectors of every mode after ``steps`` steps (homogeneous eps and
    conductivity sigma, mu0).  modes: iterable of (m, n, p, c0) with c0 the
    initial 6-vector (Ex, Ey, Ez, Hx, Hy, Hz)."""
    out = []
    for m, n, p, c0 in modes:
        A, B = mode_operators(grid, m, n, p, eps=eps, sigma=sigma)
        G = amplification(scheme, dt, A, B)
        c = np.asarray(c0, dtype=np.float64)
        for _ in range(steps):
            c = G @ c
        out.append((m, n, p, c))
    return out


def fields_from_modes(grid: Grid, modal) -> dict:
    """Sum of amplitude x shape over modes, all six components."""
    from .grid import shape as comp_shape
    f = {c: np.zeros(comp_shape(c, grid.nx, grid.ny, grid.nz)) for c in ORDER}
    for m, n, p, c in modal:
        for q, comp in enumerate(ORDER):
            if c[q] != 0.0:
                f[comp] += c[q] * mode_shape(grid, comp, m, n, p)
    return f


def field_after(grid: Grid, dt: float, scheme: str, modes, steps: int, eps_r: float = 1.0,
                sigma: float = 0.0) -> dict:
    """Exact field after ``steps`` steps from an initial E that is a sum of
    cavity modes (H = 0), in a homogeneous medium (eps_r, conductivity
    sigma).  modes: objects with m, n, p, amp, pol (the workload generator's
    records)."""
    init = [(md.m, md.n, md.p, np.array([md.amp * md.pol[0], md.amp * md.pol[1], md.amp * md.pol[2], 0, 0, 0]))
            for md in modes]
    return fields_from_modes(grid, evolve_modes(grid, dt, scheme, init, steps, eps=EPS0 * eps_r, sigma=sigma))
