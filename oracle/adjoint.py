"""Discrete adjoint of FADI for a probe-energy objective (FP64, test
infrastructure).

Objective: J(eps_r) = sum over steps n = 1..Nt and over the probe E samples
of (u_E^n)^2, where u^n is the FADI output field of step n, u_E^n = w_B / 2
with w_B the B-procedure solve of that step (Eq. 9 with Eqs. 8c-8d).  The
parameter is the relative permittivity of every cell; eps at an E sample is
eps0 times the mean over the cells sharing the edge.

The gradient is the exact reverse of the oracle's forward computation
(``schemes.fadi_init``, ``schemes.procedure``): every procedure is

    r = E + sgn b D_h H            (b = h/(2 eps) at the E sample, Eq. 36)
    T w = r,  T = 1/2 I - 1/2 b Lam     (Lam: d-weighted second difference)
    H' = H + sgn d D_e w
    E' = w - E + post

and its reverse, for adjoints (E'bar, H'bar) and a direct objective term g on
w, is

    wbar = E'bar + g + sgn D_e^T (d H'bar)
    rbar = T^{-T} wbar                 (tridiagonal, transposed coefficients)
    Ebar = rbar - E'bar
    Hbar = H'bar + sgn D_h^T (b rbar)
    bbar = rbar (sgn D_h H + 1/2 Lam w),   epsbar += -bbar b / eps
    post = (h/2) f, f = -J/(area eps) at the source: epsbar_src += E'bar_src (-post/eps)

Nothing here is blocked, scaled or fused; the pins in tests/test_oracle_adjoint.py
are central finite differences of the forward objective and the transpose
identity <lam, P x> = <P^T lam, x>.
"""
from __future__ import annotations

import numpy as np

from .grid import (AXIS, COMPS, E_COMPS, EPS0, PAIRS, apply_op, diff_e_to_h, diff_h_to_e,
                   line_operator_coeffs)
from .schemes import Problem, fadi_init, procedure
from .tridiag import thomas


# ---------------------------------------------------------------------------
# Transposes of the linear building blocks
# ---------------------------------------------------------------------------

def diff_e_to_h_T(g: np.ndarray, axis: int, spacing: float, e_shape) -> np.ndarray:
    """Transpose of ``diff_e_to_h``: (D^T g)[j] = (g[j-1] - g[j]) / d, with
    g[-1] = g[n] = 0, on the E shape (n + 1 nodes along ``axis``)."""
    out = np.zeros(e_shape)
    n = e_shape[axis] - 1
    src = [slice(None)] * 3
    tgt = [slice(None)] * 3
    src[axis] = slice(0, n)
    tgt[axis] = slice(1, n + 1)
    out[tuple(tgt)] += g[tuple(src)] / spacing
    tgt[axis] = slice(0, n)
    out[tuple(tgt)] -= g[tuple(src)] / spacing
    return out


def diff_h_to_e_T(x: np.ndarray, axis: int, spacing: float, h_shape) -> np.ndarray:
    """Transpose of ``diff_h_to_e``: the forward maps H faces f = 0..n-1 to the
    interior nodes j = 1..n-1 as (H[j] - H[j-1]) / d."""
    out = np.zeros(h_shape)
    n = x.shape[axis] - 1
    src = [slice(None)] * 3
    tgt = [slice(None)] * 3
    src[axis] = slice(1, n)
    tgt[axis] = slice(1, n)
    out[tuple(tgt)] += x[tuple(src)] / spacing
    tgt[axis] = slice(0, n - 1)
    out[tuple(tgt)] -= x[tuple(src)] / spacing
    return out


def solve_lines_T(alpha: float, lower, centre, upper, rhs_e: np.ndarray, axis: int) -> np.ndarray:
    """Solve the transpose of the ``grid.solve_lines`` system: row j of the
    forward matrix is (-lower_j, alpha - centre_j, -upper_j) at columns
    (j-1, j, j+1); the transpose has (-upper_{j-1}, alpha - centre_j,
    -lower_{j+1})."""
    r = np.moveaxis(rhs_e, axis, -1)
    lo_t = np.zeros_like(lower)
    up_t = np.zeros_like(upper)
    lo_t[..., 1:] = upper[..., :-1]
    up_t[..., :-1] = lower[..., 1:]
    x = thomas(-lo_t, alpha - centre, -up_t, r[..., 1:-1])
    w = np.zeros_like(r)
    w[..., 1:-1] = x
    return np.moveaxis(w, -1, axis)


def second_difference(d: np.ndarray, w: np.ndarray, axis: int, spacing: float, e_shape) -> np.ndarray:
    """Lam w = [d_{j+1/2}(w_{j+1} - w_j) - d_{j-1/2}(w_j - w_{j-1})] / s^2 at the
    interior nodes (zero on the two end nodes)."""
    lo, ce, up = line_operator_coeffs(np.ones(e_shape), d, axis, spacing)
    wl = np.moveaxis(w, axis, -1)
    out = np.zeros_like(wl)
    out[..., 1:-1] = lo * wl[..., :-2] + ce * wl[..., 1:-1] + up * wl[..., 2:]
    return np.moveaxis(out, -1, axis)


# ---------------------------------------------------------------------------
# Objective
# ---------------------------------------------------------------------------

def probe_masks(grid, block) -> dict:
    """1 at every E sample whose array index (i, j, k) lies in the cell block
    [i0, i1) x [j0, j1) x [k0, k1), for each E component."""
    i0, i1, j0, j1, k0, k1 = block
    out = {}
    for c in E_COMPS:
        m = np.zeros(grid.shape(c))
        m[k0:k1, j0:j1, i0:i1] = 1.0
        out[c] = m * grid.e_interior_mask(c)
    return out


def forward(P: Problem, u0: dict, steps: int, masks: dict, keep: bool = False):
    """Run FADI; returns J and (when ``keep``) every step's (v, vh, w_A, w_B)."""
    v = fadi_init(P, u0)
    J = 0.0
    tape = []
    dt = P.dt
    for n in range(steps):
        fa = P.f((n + 0.5) * dt)
        fb = P.f((n + 1.5) * dt)
        vh, wA, _ = procedure(P, v, "A", dt, post_src=None if fa is None else {c: fa[c] * dt / 2 for c in COMPS})
        v1, wB, _ = procedure(P, vh, "B", dt, post_src=None if fb is None else {c: fb[c] * dt / 2 for c in COMPS})
        for c in E_COMPS:
            J += float(np.sum(masks[c] * (0.5 * wB[c]) ** 2))
        if keep:
            tape.append((v, vh, wA, wB))
        v = v1
    return J, tape


def procedure_adjoint(P: Problem, op: str, h: float, state: dict, w: dict, lam: dict, g: dict | None,
                      post_t: float | None, epsbar: dict):
    """Reverse of ``schemes.procedure`` (no rhs source).  ``state`` is the
    procedure's input, ``w`` its solves, ``lam`` the adjoint of its output;
    returns the adjoint of its input and adds to ``epsbar`` (per E sample).
    ``post_t``: the time of the source added after the subtraction, or None."""
    grid = P.grid
    out = {c: lam[c].copy() for c in COMPS}
    for ec, hc, ax, sgn in PAIRS[op]:
        a = AXIS[ax]
        sp = grid.spacing[ax]
        mask = grid.e_interior_mask(ec)
        b = h / (2.0 * P.mat[ec])
        d = h / (2.0 * P.mat[hc])
        wbar = lam[ec] + (0.0 if g is None else g[ec])
        wbar = (wbar + sgn * diff_e_to_h_T(d * lam[hc], a, sp, grid.shape(ec))) * mask
        lo, ce, up = line_operator_coeffs(b, d, a, sp)
        rbar = solve_lines_T(0.5, 0.5 * lo, 0.5 * ce, 0.5 * up, wbar, a) * mask
        out[ec] = (rbar - lam[ec]) * mask
        out[hc] = lam[hc] + sgn * diff_h_to_e_T(b * rbar, a, sp, grid.shape(hc))
        dh = diff_h_to_e(state[hc], a, sp, grid.shape(ec))
        lam_w = second_difference(d, w[ec], a, sp, grid.shape(ec))
        bbar = rbar * (sgn * dh + 0.5 * lam_w)
        epsbar[ec] += -bbar * b / P.mat[ec]
    if post_t is not None and P.source is not None:
        f = P.f(post_t)
        s = P.source
        c = s.comp
        post = 0.5 * P.dt * f[c][s.k, s.j, s.i]
        epsbar[c][s.k, s.j, s.i] += lam[c][s.k, s.j, s.i] * (-post / P.mat[c][s.k, s.j, s.i])
    return out


def init_adjoint(P: Problem, u0: dict, lam0: dict, epsbar: dict):
    """Reverse of ``schemes.fadi_init`` with respect to eps:
    v^0 = u^0 + (dt/2) B u^0 + (dt/2) f(dt/2); the E rows of B u^0 carry 1/eps."""
    Bu = apply_op(P.grid, P.mat, "B", u0)
    for c in E_COMPS:
        epsbar[c] += lam0[c] * (-0.5 * P.dt * Bu[c] / P.mat[c])
    if P.source is not None:
        s = P.source
        c = s.comp
        post = 0.5 * P.dt * P.f(0.5 * P.dt)[c][s.k, s.j, s.i]
        epsbar[c][s.k, s.j, s.i] += lam0[c][s.k, s.j, s.i] * (-post / P.mat[c][s.k, s.j, s.i])


def cell_gradient(grid, epsbar: dict) -> np.ndarray:
    """Chain rule through the edge averaging of ``grid.material_at_samples``:
    eps_sample = eps0 * mean of its in-domain cells, so each cell receives
    eps0 * epsbar_sample / (number of in-domain cells of that sample)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    g = np.zeros((nz + 2, ny + 2, nx + 2))      # cells padded by one on every side
    cnt = np.zeros((nz + 2, ny + 2, nx + 2))
    cnt[1:-1, 1:-1, 1:-1] = 1.0
    # (component, offsets of the cells sharing the sample in padded coordinates)
    spec = {
        # Ex (i+1/2, j, k): cells (i, j-1..j, k-1..k) -> padded (k+dk, j+dj, i+1), dk, dj in {0, 1}
        "ex": [(dk, dj, 1) for dk in (0, 1) for dj in (0, 1)],
        # Ey (i, j+1/2, k): cells (i-1..i, j, k-1..k)
        "ey": [(dk, 1, di) for dk in (0, 1) for di in (0, 1)],
        # Ez (i, j, k+1/2): cells (i-1..i, j-1..j, k)
        "ez": [(1, dj, di) for dj in (0, 1) for di in (0, 1)],
    }
    for c, offs in spec.items():
        sh = grid.shape(c)
        n = sum(cnt[o[0]:o[0] + sh[0], o[1]:o[1] + sh[1], o[2]:o[2] + sh[2]] for o in offs)
        share = np.where(n > 0, EPS0 * epsbar[c] / np.maximum(n, 1.0), 0.0)
        for o in offs:
            g[o[0]:o[0] + sh[0], o[1]:o[1] + sh[1], o[2]:o[2] + sh[2]] += share
    return g[1:-1, 1:-1, 1:-1]


def gradient(P: Problem, u0: dict, steps: int, masks: dict):
    """(J, dJ/d eps_r per cell, dJ/d eps per E sample) by the discrete adjoint."""
    J, tape = forward(P, u0, steps, masks, keep=True)
    grid = P.grid
    dt = P.dt
    lam = {c: np.zeros(grid.shape(c)) for c in COMPS}
    epsbar = {c: np.zeros(grid.shape(c)) for c in E_COMPS}
    src = P.source is not None
    for n in range(steps - 1, -1, -1):
        v, vh, wA, wB = tape[n]
        g = {c: masks[c] * 0.5 * wB[c] for c in E_COMPS}
        lam = procedure_adjoint(P, "B", dt, vh, wB, lam, g, (n + 1.5) * dt if src else None, epsbar)
        lam = procedure_adjoint(P, "A", dt, v, wA, lam, None, (n + 0.5) * dt if src else None, epsbar)
    init_adjoint(P, u0, lam, epsbar)
    return J, cell_gradient(grid, epsbar), epsbar
