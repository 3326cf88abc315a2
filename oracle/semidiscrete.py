"""The semi-discrete Yee system integrated in time by classic RK4 (FP64).

TEST INFRASTRUCTURE ONLY (part of the oracle).

Every splitting scheme of Sec. II approximates, in time, the same
semi-discrete system: Maxwell's curl equations on the Yee grid (the
operator A + B of Eqs. 33-34, PEC walls) driven by a current density,

    d/dt E = (1/eps) curl H - J/eps,      d/dt H = -(1/mu) curl E.

A current I(t) flowing along one E sample spreads over that sample's
dual face, J = I / area, so the forcing sits on that one E sample.  This
module integrates the system with the explicit four-stage Runge-Kutta
method at a small step, which makes its time error negligible next to
that of the implicit schemes.  It touches none of the schemes' source
bookkeeping: the forcing is formed here from the current and the medium,
so a wrong source weight or a wrong sampling time inside the schemes shows
up as a failure to converge to this solution as dt -> 0 (first order for
LOD1/FLOD, second order for ADI/FADI and SS2/FSS, Table I).
"""
from __future__ import annotations

import math

import numpy as np

from .grid import COMPS, Grid, apply_op


def forcing(grid: Grid, mat: dict, source, t: float) -> dict:
    """-J/eps at time t: nonzero only at the source's E sample, where
    J = I(t) / (area of the sample's dual face)."""
    out = {c: np.zeros(grid.shape(c)) for c in COMPS}
    if source is None:
        return out
    area = {"ex": grid.dy * grid.dz, "ey": grid.dx * grid.dz, "ez": grid.dx * grid.dy}[source.comp]
    eps = mat[source.comp][source.k, source.j, source.i]
    out[source.comp][source.k, source.j, source.i] = -float(source.current(t)) / (area * eps)
    return out


def rhs(grid: Grid, mat: dict, source, u: dict, t: float) -> dict:
    """(A + B) u - J/eps, with the PEC walls of A and B."""
    a = apply_op(grid, mat, "A", u)
    b = apply_op(grid, mat, "B", u)
    f = forcing(grid, mat, source, t)
    return {c: a[c] + b[c] + f[c] for c in COMPS}


def rk4(grid: Grid, mat: dict, source, u0: dict, t_end: float, steps: int, t0: float = 0.0) -> dict:
    """u(t0 + t_end) from u(t0) = u0 by ``steps`` classic RK4 steps of t_end/steps."""
    h = t_end / steps
    u = {c: np.array(u0[c], dtype=np.float64, copy=True) for c in COMPS}
    for n in range(steps):
        t = t0 + n * h
        k1 = rhs(grid, mat, source, u, t)
        k2 = rhs(grid, mat, source, {c: u[c] + 0.5 * h * k1[c] for c in COMPS}, t + 0.5 * h)
        k3 = rhs(grid, mat, source, {c: u[c] + 0.5 * h * k2[c] for c in COMPS}, t + 0.5 * h)
        k4 = rhs(grid, mat, source, {c: u[c] + h * k3[c] for c in COMPS}, t + h)
        u = {c: u[c] + (h / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]) for c in COMPS}
    return u


def rk4_stable_steps(grid: Grid, t_end: float, cfl: float = 0.25) -> int:
    """Steps that keep RK4 at ``cfl`` times the explicit Yee limit (the
    skew-adjoint spectrum of A + B lies within +-2/dt_CFL, and RK4 is stable
    on the imaginary axis up to 2.83/h)."""
    return max(1, int(math.ceil(t_end / (cfl * grid.dt_cfl()))))
