"""Yee grid, materials and the Maxwell splitting operators of the oracle.

Sec. III of the paper: lossless isotropic medium, u = (Ex, Ey, Ez, Hx, Hy, Hz),
splitting operators A (Eq. 33) and B (Eq. 34) built from first differences
d_x, d_y, d_z, and b = dt/(2 eps), d = dt/(2 mu) (Eq. 36).

Lossy media (the paper assumes a lossless medium when it writes A and B;
its splitting formulae of Sec. II hold for any linear operators): an
electric conductivity sigma adds -sigma/eps E to dE/dt.  That diagonal term
is split evenly between the two operators, A_s = A - (1/2) diag(sigma/eps)
and B_s = B - (1/2) diag(sigma/eps) on the E rows, so that every E
component, which has one line pair in A and one in B, loses half in each
procedure.  In a procedure of length h the implicit diagonal becomes
1/2 + b sigma / 4 (b = h / (2 eps)).

Higher-order differences (the paper names "higher order, parameter
optimized, compact" difference operators as possible variants without
formulae, end of Sec. III-A): with order = 4 every first difference of A and
B is the fourth-order staggered central difference
    (9/8 (u_{+1/2} - u_{-1/2}) - 1/24 (u_{+3/2} - u_{-3/2})) / d,
and the points past a PEC wall are images: tangential E is odd about the
wall (E_{-j} = -E_j), the H samples half a cell off it are even
(H_{-1/2-f} = H_{1/2+f}).  The two differences stay exact negative
transposes of each other, so A and B stay skew in the energy product and
every scheme keeps its invariant; eliminating H gives line systems of
bandwidth 3, which the oracle solves densely line by line.

Readings of what the paper leaves open (each is a documented choice):
* differences are the standard Yee second-order central differences between
  staggered samples (sample layout in ``workloads``);
* the walls are perfect electric conductors: tangential E samples on the six
  walls are fixed at zero and are not unknowns;
* for inhomogeneous media, eps at an E sample is the mean of the (up to four)
  cells sharing that edge, mu at an H sample the mean of the (up to two)
  cells sharing that face; eliminating H then gives (b_j/2) d(d d w) with b at
  the E sample and d at the H faces, which reduces to the paper's (bd/2) d^2
  for a homogeneous medium.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .tridiag import thomas

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)

E_COMPS = ("ex", "ey", "ez")
H_COMPS = ("hx", "hy", "hz")
COMPS = E_COMPS + H_COMPS
AXIS = {"x": 2, "y": 1, "z": 0}          # array axis of each direction ([k, j, i] layout)

# The three (E, H, line axis, sign) pairs of each operator.  A (Eq. 33) holds
# +(1/eps) d_y Hz, +(1/eps) d_z Hx, +(1/eps) d_x Hy in its E rows and
# +(1/mu) d_z Ey, +(1/mu) d_x Ez, +(1/mu) d_y Ex in its H rows; B (Eq. 34)
# holds the other half of the curls with a minus sign.
PAIRS = {
    "A": (("ex", "hz", "y", +1.0), ("ey", "hx", "z", +1.0), ("ez", "hy", "x", +1.0)),
    "B": (("ex", "hy", "z", -1.0), ("ey", "hz", "x", -1.0), ("ez", "hx", "y", -1.0)),
}


def shape(comp, nx, ny, nz):
    return {
        "ex": (nz + 1, ny + 1, nx), "ey": (nz + 1, ny, nx + 1), "ez": (nz, ny + 1, nx + 1),
        "hx": (nz, ny, nx + 1), "hy": (nz, ny + 1, nx), "hz": (nz + 1, ny, nx),
    }[comp]


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    order: int = 2          # 2: Yee differences; 4: fourth-order staggered differences

    @property
    def spacing(self):
        return {"x": self.dx, "y": self.dy, "z": self.dz}

    def shape(self, comp):
        return shape(comp, self.nx, self.ny, self.nz)

    def zeros(self):
        return {c: np.zeros(self.shape(c)) for c in COMPS}

    def dt_cfl(self) -> float:
        """Explicit-Yee stability limit 1/(c0 sqrt(sum 1/d^2)) over the active
        directions (x, y only when nz == 1)."""
        s = 1.0 / self.dx ** 2 + 1.0 / self.dy ** 2
        if self.nz > 1:
            s += 1.0 / self.dz ** 2
        return 1.0 / (C0 * math.sqrt(s))

    def cell_volume(self) -> float:
        return self.dx * self.dy * self.dz

    # -- PEC -----------------------------------------------------------------
    def e_interior_mask(self, comp) -> np.ndarray:
        """1 where an E sample is an unknown, 0 on the walls (tangential E)."""
        m = np.ones(self.shape(comp))
        if comp == "ex":
            m[:, 0, :] = 0; m[:, -1, :] = 0; m[0] = 0; m[-1] = 0
        elif comp == "ey":
            m[:, :, 0] = 0; m[:, :, -1] = 0; m[0] = 0; m[-1] = 0
        elif comp == "ez":
            m[:, :, 0] = 0; m[:, :, -1] = 0; m[:, 0, :] = 0; m[:, -1, :] = 0
        return m


# ---------------------------------------------------------------------------
# Materials
# ---------------------------------------------------------------------------

def _avg(cells: np.ndarray, pad: tuple, windows) -> np.ndarray:
    """Mean of the in-domain cells in each window.  ``pad`` pads the cell
    array by one on the axes flagged; ``windows`` lists the slices to add."""
    padw = [(1, 1) if p else (0, 0) for p in pad]
    val = np.pad(cells, padw)
    cnt = np.pad(np.ones_like(cells), padw)
    s = sum(val[w] for w in windows)
    n = sum(cnt[w] for w in windows)
    return s / n


def material_at_samples(grid: Grid, eps_r_cell=None, mu_r_cell=None, sigma_cell=None) -> dict:
    """Absolute eps at every E sample and mu at every H sample; with a
    per-cell conductivity [S/m], also mat["sigma"][ec] at every E sample (the
    mean of the in-domain cells sharing the edge, as for eps)."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    er = np.ones((nz, ny, nx)) if eps_r_cell is None else np.asarray(eps_r_cell, dtype=np.float64)
    mr = np.ones((nz, ny, nx)) if mu_r_cell is None else np.asarray(mu_r_cell, dtype=np.float64)
    b = slice(None)
    out = {}
    # Ex edge (i+1/2, j, k): cells (i, j-1..j, k-1..k)
    out["ex"] = EPS0 * _avg(er, (1, 1, 0), [(slice(0, nz + 1), slice(0, ny + 1), b),
                                            (slice(1, nz + 2), slice(0, ny + 1), b),
                                            (slice(0, nz + 1), slice(1, ny + 2), b),
                                            (slice(1, nz + 2), slice(1, ny + 2), b)])
    # Ey edge (i, j+1/2, k): cells (i-1..i, j, k-1..k)
    out["ey"] = EPS0 * _avg(er, (1, 0, 1), [(slice(0, nz + 1), b, slice(0, nx + 1)),
                                            (slice(1, nz + 2), b, slice(0, nx + 1)),
                                            (slice(0, nz + 1), b, slice(1, nx + 2)),
                                            (slice(1, nz + 2), b, slice(1, nx + 2))])
    # Ez edge (i, j, k+1/2): cells (i-1..i, j-1..j, k)
    out["ez"] = EPS0 * _avg(er, (0, 1, 1), [(b, slice(0, ny + 1), slice(0, nx + 1)),
                                            (b, slice(1, ny + 2), slice(0, nx + 1)),
                                            (b, slice(0, ny + 1), slice(1, nx + 2)),
                                            (b, slice(1, ny + 2), slice(1, nx + 2))])
    if sigma_cell is not None:
        sg = np.asarray(sigma_cell, dtype=np.float64)
        out["sigma"] = {
            "ex": _avg(sg, (1, 1, 0), [(slice(0, nz + 1), slice(0, ny + 1), b), (slice(1, nz + 2), slice(0, ny + 1), b),
                                      (slice(0, nz + 1), slice(1, ny + 2), b), (slice(1, nz + 2), slice(1, ny + 2), b)]),
            "ey": _avg(sg, (1, 0, 1), [(slice(0, nz + 1), b, slice(0, nx + 1)), (slice(1, nz + 2), b, slice(0, nx + 1)),
                                      (slice(0, nz + 1), b, slice(1, nx + 2)), (slice(1, nz + 2), b, slice(1, nx + 2))]),
            "ez": _avg(sg, (0, 1, 1), [(b, slice(0, ny + 1), slice(0, nx + 1)), (b, slice(1, ny + 2), slice(0, nx + 1)),
                                      (b, slice(0, ny + 1), slice(1, nx + 2)), (b, slice(1, ny + 2), slice(1, nx + 2))]),
        }
    # Hx face (i, j+1/2, k+1/2): cells (i-1..i, j, k)
    out["hx"] = MU0 * _avg(mr, (0, 0, 1), [(b, b, slice(0, nx + 1)), (b, b, slice(1, nx + 2))])
    # Hy face (i+1/2, j, k+1/2): cells (i, j-1..j, k)
    out["hy"] = MU0 * _avg(mr, (0, 1, 0), [(b, slice(0, ny + 1), b), (b, slice(1, ny + 2), b)])
    # Hz face (i+1/2, j+1/2, k): cells (i, j, k-1..k)
    out["hz"] = MU0 * _avg(mr, (1, 0, 0), [(slice(0, nz + 1), b, b), (slice(1, nz + 2), b, b)])
    return out


# ---------------------------------------------------------------------------
# First differences between staggered samples
# ---------------------------------------------------------------------------

def diff_h_to_e(h: np.ndarray, axis: int, spacing: float, e_shape) -> np.ndarray:
    """d/d(eta) of an H component at the E samples: (H[j] - H[j-1]) / d for
    the interior E nodes j = 1..N-1 along ``axis``; zero at the two end nodes
    (the PEC mask later zeroes every wall sample anyway)."""
    out = np.zeros(e_shape)
    n = e_shape[axis] - 1          # number of cells along the line
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    tgt = [slice(None)] * 3
    hi[axis] = slice(1, n)
    lo[axis] = slice(0, n - 1)
    tgt[axis] = slice(1, n)
    out[tuple(tgt)] = (h[tuple(hi)] - h[tuple(lo)]) / spacing
    return out


def diff_e_to_h(e: np.ndarray, axis: int, spacing: float) -> np.ndarray:
    """d/d(eta) of an E component at the H samples: (E[j+1] - E[j]) / d."""
    hi = [slice(None)] * 3
    lo = [slice(None)] * 3
    hi[axis] = slice(1, None)
    lo[axis] = slice(0, -1)
    return (e[tuple(hi)] - e[tuple(lo)]) / spacing


C4 = (9.0 / 8.0, -1.0 / 24.0)   # fourth-order staggered difference weights


def _pad_images(x: np.ndarray, axis: int, odd: bool) -> np.ndarray:
    """x with one image sample added before and after along ``axis``: for E
    (odd about the walls, which are its first and last samples) x[-1] = -x[1]
    and x[n+1] = -x[n-1]; for H (even, half a cell off the walls) x[-1] = x[0]
    and x[n] = x[n-1]."""
    n = x.shape[axis]
    idx_lo = 1 if odd else 0
    idx_hi = n - 2 if odd else n - 1
    lo = np.take(x, [idx_lo], axis=axis)
    hi = np.take(x, [idx_hi], axis=axis)
    if odd:
        lo, hi = -lo, -hi
    return np.concatenate([lo, x, hi], axis=axis)


def diff_e_to_h4(e: np.ndarray, axis: int, spacing: float) -> np.ndarray:
    """Fourth-order d/d(eta) of an E component at the H samples (faces
    f = 0..n-1 between nodes f and f+1), PEC images past the walls."""
    ep = _pad_images(e, axis, odd=True)        # ep[j + 1] = E_j
    n = e.shape[axis] - 1

    def sl(a, b):
        s = [slice(None)] * e.ndim
        s[axis] = slice(a, b)
        return tuple(s)
    c1, c2 = C4
    return (c1 * (ep[sl(2, n + 2)] - ep[sl(1, n + 1)]) + c2 * (ep[sl(3, n + 3)] - ep[sl(0, n)])) / spacing


def diff_h_to_e4(h: np.ndarray, axis: int, spacing: float, e_shape) -> np.ndarray:
    """Fourth-order d/d(eta) of an H component at the E nodes j = 1..n-1
    (zero at the two wall nodes), PEC images past the walls."""
    hp = _pad_images(h, axis, odd=False)       # hp[f + 1] = H_f
    n = e_shape[axis] - 1
    out = np.zeros(e_shape)
    if n < 2:
        return out

    def sl(a, b):
        s = [slice(None)] * h.ndim
        s[axis] = slice(a, b)
        return tuple(s)
    c1, c2 = C4
    tgt = [slice(None)] * len(e_shape)
    tgt[axis] = slice(1, n)
    # node j (1..n-1): faces j, j-1, j+1, j-2 at hp[j+1], hp[j], hp[j+2], hp[j-1]
    out[tuple(tgt)] = (c1 * (hp[sl(2, n + 1)] - hp[sl(1, n)]) + c2 * (hp[sl(3, n + 2)] - hp[sl(0, n - 1)])) / spacing
    return out


def d_e_to_h(grid: Grid, e, axis, spacing):
    return diff_e_to_h4(e, axis, spacing) if grid.order == 4 else diff_e_to_h(e, axis, spacing)


def d_h_to_e(grid: Grid, h, axis, spacing, e_shape):
    return diff_h_to_e4(h, axis, spacing, e_shape) if grid.order == 4 else diff_h_to_e(h, axis, spacing, e_shape)


def line_matrices4(n: int, spacing: float):
    """The fourth-order differences of one line as matrices over its
    interior E nodes 1..n-1: DEH (faces x interior nodes) and DHE (interior
    nodes x faces), built by applying the difference functions to unit
    vectors (images included)."""
    m = max(n - 1, 0)
    DEH = np.zeros((n, m))
    DHE = np.zeros((m, n))
    for k in range(m):
        e = np.zeros(n + 1)
        e[k + 1] = 1.0
        DEH[:, k] = diff_e_to_h4(e, 0, spacing)
    for f in range(n):
        h = np.zeros(n)
        h[f] = 1.0
        DHE[:, f] = diff_h_to_e4(h, 0, spacing, (n + 1,))[1:n]
    return DEH, DHE


def solve_lines4(diag, gE: np.ndarray, gH: np.ndarray, rhs_e: np.ndarray, axis: int, spacing: float) -> np.ndarray:
    """Solve diag*w - gE * DHE (gH * DEH w) = rhs along ``axis`` (fourth-order
    differences) for the interior nodes, one dense system per line; w = 0 on
    the two wall nodes.  diag is a number or an array of the E shape."""
    r = np.moveaxis(rhs_e, axis, -1)
    n = r.shape[-1] - 1
    w = np.zeros_like(r)
    if n < 2:
        return np.moveaxis(w, -1, axis)
    DEH, DHE = line_matrices4(n, spacing)
    ge = np.moveaxis(gE, axis, -1)[..., 1:-1]
    gh = np.moveaxis(gH, axis, -1)
    dg = np.moveaxis(diag, axis, -1)[..., 1:-1] if np.ndim(diag) else np.full(ge.shape, float(diag))
    K = np.einsum("jf,...f,fk->...jk", DHE, gh, DEH)
    M = -ge[..., :, None] * K
    idx = np.arange(n - 1)
    M[..., idx, idx] += dg
    w[..., 1:-1] = np.linalg.solve(M, r[..., 1:-1, None])[..., 0]
    return np.moveaxis(w, -1, axis)


def apply_op(grid: Grid, mat: dict, op: str, u: dict) -> dict:
    """O u for O = A (Eq. 33) or B (Eq. 34), PEC walls applied; in a lossy
    medium each operator also carries -(1/2)(sigma/eps) E on its E rows."""
    out = {c: np.zeros(grid.shape(c)) for c in COMPS}
    for ec, hc, ax, sgn in PAIRS[op]:
        a = AXIS[ax]
        sp = grid.spacing[ax]
        out[ec] += sgn * d_h_to_e(grid, u[hc], a, sp, grid.shape(ec)) / mat[ec]
        out[hc] += sgn * d_e_to_h(grid, u[ec], a, sp) / mat[hc]
        if "sigma" in mat:
            out[ec] -= 0.5 * mat["sigma"][ec] / mat[ec] * u[ec]
    for ec in E_COMPS:
        out[ec] *= grid.e_interior_mask(ec)
    return out


def add(u: dict, v: dict, alpha: float = 1.0) -> dict:
    return {c: u[c] + alpha * v[c] for c in u}


def scale(u: dict, alpha: float) -> dict:
    return {c: alpha * u[c] for c in u}


# ---------------------------------------------------------------------------
# Tridiagonal line systems
# ---------------------------------------------------------------------------

def line_operator_coeffs(gE: np.ndarray, gH: np.ndarray, axis: int, spacing: float):
    """Coefficients of the line operator w -> gE_j * [gH_{j+1/2}(w_{j+1}-w_j)
    - gH_{j-1/2}(w_j - w_{j-1})] / d^2 at the interior nodes j = 1..N-1, with
    the system axis moved last.  Returns (lower, centre, upper) such that the
    operator is lower*w_{j-1} + centre*w_j + upper*w_{j+1}."""
    ge = np.moveaxis(gE, axis, -1)[..., 1:-1]
    gh = np.moveaxis(gH, axis, -1)
    gm = gh[..., :-1]             # face j-1/2 of node j (j = 1..N-1)
    gp = gh[..., 1:]              # face j+1/2
    s2 = spacing * spacing
    lower = ge * gm / s2
    upper = ge * gp / s2
    centre = -(lower + upper)
    return lower, centre, upper


def solve_lines(alpha, lower, centre, upper, rhs_e: np.ndarray, axis: int) -> np.ndarray:
    """Solve alpha*w - (lower, centre, upper)-operator w = rhs along ``axis``
    for the interior nodes; w = 0 on the two end nodes (PEC).  alpha is a
    number or an array of the E component's shape (one diagonal per node)."""
    r = np.moveaxis(rhs_e, axis, -1)
    if np.ndim(alpha):
        alpha = np.moveaxis(alpha, axis, -1)[..., 1:-1]
    x = thomas(-lower, alpha - centre, -upper, r[..., 1:-1])
    w = np.zeros_like(r)
    w[..., 1:-1] = x
    return np.moveaxis(w, -1, axis)


def solve_implicit(grid: Grid, mat: dict, op: str, tau: float, rhs: dict) -> dict:
    """Solve (I - tau*O) u = rhs for O = A or B, by eliminating H pair by pair.

    For a pair with E row  E - sgn*(tau/eps) d(H) = rE  and H row
    H - sgn*(tau/mu) d(E) = rH, substituting H = rH + sgn*(tau/mu) d(E) gives
    the tridiagonal line system E - (tau/eps) d((tau/mu) d E) = rE + sgn*(tau/eps) d(rH);
    H is then recovered explicitly.  In a lossy medium the E row's diagonal
    is 1 + tau sigma / (2 eps).  tau may be negative."""
    out = {}
    for ec, hc, ax, sgn in PAIRS[op]:
        a = AXIS[ax]
        sp = grid.spacing[ax]
        mask = grid.e_interior_mask(ec)
        gE = tau / mat[ec]
        gH = tau / mat[hc]
        rE = (rhs[ec] + sgn * gE * d_h_to_e(grid, rhs[hc], a, sp, grid.shape(ec))) * mask
        alpha = 1.0 + 0.5 * tau * mat["sigma"][ec] / mat[ec] if "sigma" in mat else 1.0
        if grid.order == 4:
            w = solve_lines4(alpha, gE, gH, rE, a, sp) * mask
        else:
            lo, ce, up = line_operator_coeffs(gE, gH, a, sp)
            w = solve_lines(alpha, lo, ce, up, rE, a) * mask
        out[ec] = w
        out[hc] = rhs[hc] + sgn * gH * d_e_to_h(grid, w, a, sp)
    return out
