"""Brute-force dense operators for tiny grids (a pin for the structured oracle).

A and B of Eqs. 33-34 are assembled entry by entry with explicit loops over
the Yee samples, as (6 components flattened) x (6 components flattened)
matrices; the original splitting formulae are then applied with dense
``numpy.linalg.solve``.  Rows of tangential wall E samples are zero (PEC), so
those samples stay at their initial value 0.
"""
from __future__ import annotations

import numpy as np

from .grid import COMPS, Grid


def layout(grid: Grid):
    off = {}
    n = 0
    for c in COMPS:
        off[c] = n
        sk, sj, si = grid.shape(c)
        n += sk * sj * si
    return off, n


def to_vec(grid: Grid, u: dict) -> np.ndarray:
    return np.concatenate([u[c].ravel() for c in COMPS])


def from_vec(grid: Grid, x: np.ndarray) -> dict:
    off, _ = layout(grid)
    out = {}
    for c in COMPS:
        sh = grid.shape(c)
        out[c] = x[off[c]: off[c] + sh[0] * sh[1] * sh[2]].reshape(sh).copy()
    return out


def assemble(grid: Grid, mat: dict):
    """Dense A (Eq. 33) and B (Eq. 34) (with the split loss diagonal in a
    lossy medium)."""
    off, n = layout(grid)
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    dx, dy, dz = grid.dx, grid.dy, grid.dz
    A = np.zeros((n, n))
    B = np.zeros((n, n))

    def idx(c, k, j, i):
        sk, sj, si = grid.shape(c)
        return off[c] + (k * sj + j) * si + i

    def loop(c):
        sk, sj, si = grid.shape(c)
        for k in range(sk):
            for j in range(sj):
                for i in range(si):
                    yield k, j, i

    for k, j, i in loop("ex"):
        if 1 <= j <= ny - 1 and 1 <= k <= nz - 1:
            r = idx("ex", k, j, i); e = mat["ex"][k, j, i]
            A[r, idx("hz", k, j, i)] += 1 / (e * dy); A[r, idx("hz", k, j - 1, i)] -= 1 / (e * dy)
            B[r, idx("hy", k, j, i)] -= 1 / (e * dz); B[r, idx("hy", k - 1, j, i)] += 1 / (e * dz)
    for k, j, i in loop("ey"):
        if 1 <= i <= nx - 1 and 1 <= k <= nz - 1:
            r = idx("ey", k, j, i); e = mat["ey"][k, j, i]
            A[r, idx("hx", k, j, i)] += 1 / (e * dz); A[r, idx("hx", k - 1, j, i)] -= 1 / (e * dz)
            B[r, idx("hz", k, j, i)] -= 1 / (e * dx); B[r, idx("hz", k, j, i - 1)] += 1 / (e * dx)
    for k, j, i in loop("ez"):
        if 1 <= i <= nx - 1 and 1 <= j <= ny - 1:
            r = idx("ez", k, j, i); e = mat["ez"][k, j, i]
            A[r, idx("hy", k, j, i)] += 1 / (e * dx); A[r, idx("hy", k, j, i - 1)] -= 1 / (e * dx)
            B[r, idx("hx", k, j, i)] -= 1 / (e * dy); B[r, idx("hx", k, j - 1, i)] += 1 / (e * dy)
    if "sigma" in mat:
        # lossy media: -(1/2) sigma/eps on the diagonal of every interior E
        # row, in A and in B alike
        for c, inside in (("ex", lambda k, j, i: 1 <= j <= ny - 1 and 1 <= k <= nz - 1),
                          ("ey", lambda k, j, i: 1 <= i <= nx - 1 and 1 <= k <= nz - 1),
                          ("ez", lambda k, j, i: 1 <= i <= nx - 1 and 1 <= j <= ny - 1)):
            for k, j, i in loop(c):
                if inside(k, j, i):
                    r = idx(c, k, j, i)
                    g = 0.5 * mat["sigma"][c][k, j, i] / mat[c][k, j, i]
                    A[r, r] -= g
                    B[r, r] -= g
    for k, j, i in loop("hx"):
        r = idx("hx", k, j, i); m = mat["hx"][k, j, i]
        A[r, idx("ey", k + 1, j, i)] += 1 / (m * dz); A[r, idx("ey", k, j, i)] -= 1 / (m * dz)
        B[r, idx("ez", k, j + 1, i)] -= 1 / (m * dy); B[r, idx("ez", k, j, i)] += 1 / (m * dy)
    for k, j, i in loop("hy"):
        r = idx("hy", k, j, i); m = mat["hy"][k, j, i]
        A[r, idx("ez", k, j, i + 1)] += 1 / (m * dx); A[r, idx("ez", k, j, i)] -= 1 / (m * dx)
        B[r, idx("ex", k + 1, j, i)] -= 1 / (m * dz); B[r, idx("ex", k, j, i)] += 1 / (m * dz)
    for k, j, i in loop("hz"):
        r = idx("hz", k, j, i); m = mat["hz"][k, j, i]
        A[r, idx("ex", k, j + 1, i)] += 1 / (m * dy); A[r, idx("ex", k, j, i)] -= 1 / (m * dy)
        B[r, idx("ey", k, j, i + 1)] -= 1 / (m * dx); B[r, idx("ey", k, j, i)] += 1 / (m * dx)
    return A, B


# Fourth-order assembly (Grid.order == 4): the terms of Eqs. 33-34 written
# out again, (E row, H column, line axis, sign, operator), each first
# difference being the fourth-order staggered one with PEC images.
_TERMS4 = (
    ("ex", "hz", "y", +1, "A"), ("ey", "hx", "z", +1, "A"), ("ez", "hy", "x", +1, "A"),
    ("ex", "hy", "z", -1, "B"), ("ey", "hz", "x", -1, "B"), ("ez", "hx", "y", -1, "B"),
)


def assemble4(grid: Grid, mat: dict):
    """Dense A and B with fourth-order staggered differences, entry by entry.
    E row at node j of its line: (9/8)(H_j - H_{j-1}) - (1/24)(H_{j+1} - H_{j-2});
    a face past a wall is its mirror image (H even).  H row at face f:
    (9/8)(E_{f+1} - E_f) - (1/24)(E_{f+2} - E_{f-1}); a node past a wall is
    minus its mirror image (tangential E odd)."""
    off, n = layout(grid)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    c1, c2 = 9.0 / 8.0, -1.0 / 24.0
    dims = {"x": grid.nx, "y": grid.ny, "z": grid.nz}
    sp = {"x": grid.dx, "y": grid.dy, "z": grid.dz}
    pos = {"x": 2, "y": 1, "z": 0}

    def idx(c, kji):
        sk, sj, si = grid.shape(c)
        k, j, i = kji
        return off[c] + (k * sj + j) * si + i

    def samples(c):
        sk, sj, si = grid.shape(c)
        for k in range(sk):
            for j in range(sj):
                for i in range(si):
                    yield [k, j, i]

    for ec, hc, ax, sg, op in _TERMS4:
        O = A if op == "A" else B
        N = dims[ax]
        a = pos[ax]
        d = sp[ax]
        emask = grid.e_interior_mask(ec)
        for kji in samples(ec):
            if emask[tuple(kji)] == 0:
                continue
            j = kji[a]
            r = idx(ec, kji)
            e = mat[ec][tuple(kji)]
            for fo, wgt in ((0, c1), (-1, -c1), (1, c2), (-2, -c2)):
                f = j + fo
                if f < 0:
                    f = -1 - f
                if f > N - 1:
                    f = 2 * N - 1 - f
                col = list(kji)
                col[a] = f
                O[r, idx(hc, col)] += sg * wgt / (e * d)
        for kji in samples(hc):
            f = kji[a]
            r = idx(hc, kji)
            m = mat[hc][tuple(kji)]
            for no, wgt in ((1, c1), (0, -c1), (2, c2), (-1, -c2)):
                node = f + no
                s_img = 1.0
                if node < 0:
                    node, s_img = -node, -1.0
                if node > N:
                    node, s_img = 2 * N - node, -1.0
                col = list(kji)
                col[a] = node
                if emask[tuple(col)] == 0:
                    continue         # a wall sample: fixed at zero
                O[r, idx(ec, col)] += sg * s_img * wgt / (m * d)
    return A, B


def cn(Oi, Oe, tau, x, f=None):
    """(I - tau Oi) x' = (I + tau Oe) x (+ tau f), dense."""
    I = np.eye(Oi.shape[0])
    rhs = x + tau * (Oe @ x)
    if f is not None:
        rhs = rhs + tau * f
    return np.linalg.solve(I - tau * Oi, rhs)


def adi_step(A, B, dt, x, f=None):
    return cn(B, A, dt / 2, cn(A, B, dt / 2, x, f), f)


def lod1_step(A, B, dt, x, f=None):
    return cn(B, B, dt / 2, cn(A, A, dt / 2, x, f), f)


def ss2_step(A, B, dt, x, f=None):
    x = cn(A, A, dt / 4, x, f)
    x = cn(B, B, dt / 2, x, f)
    return cn(A, A, dt / 4, x, f)
