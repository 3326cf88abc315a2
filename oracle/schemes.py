"""Original and fundamental splitting schemes of the oracle (FP64).

State and fields are dicts of the six Yee components (``[k, j, i]`` arrays).

Original schemes (Sec. II) are written straight from their splitting
formulae with the operators of Eqs. 33-34:
    ADI  Eq. 1,  LOD1 Eq. 11,  SS2 Eq. 16,  LOD2 Eqs. 18-20.
Fundamental schemes are written in the per-component form of Sec. III:
    FADI  Eqs. 7-10 with Eqs. 37-44 (fused H updates Eqs. 43-44),
    FLOD  Eq. 15, FSS Eq. 17, FLOD2 Eqs. 21-23, all with the per-component
          procedure of Eqs. 45-52 (fused H updates Eqs. 51-52).

Sources (the paper omits them, Sec. II): a current I(t) on one E sample
contributes f_E = -I(t) / (A * eps) with A the sample's dual-face area.  Each
procedure of length h adds (h/2) f(t_n + dt/2) to its original-form right-hand
side; the weights of one step sum to dt.  In fundamental form this becomes
+(h/4) f in the implicit right-hand side (FLOD, FSS) or, for FADI,
+(dt/2) f added to the auxiliary state after each procedure (it is part of
the auxiliary variable v of Eqs. 2 and 8).  Every sample of the current is
taken at a half-integer time t_n + dt/2.  LOD2 is the one exception to the
mid-step sampling: its input and output processing (Eqs. 19-20) make it a
similarity transform of Strang splitting with B on the outside, so the B
sub-step of its main loop is centred on t_{n+1} and takes the mean of the
samples at t_n + dt/2 and t_n + 3dt/2; its input and output processing,
each a quarter step that runs once, take the sample of the step that
follows them.  With these placements every scheme converges, as dt -> 0 at
a fixed time, to the semi-discrete Yee system with its current at the order
Table I gives (first for LOD1, second for ADI, SS2 and LOD2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from .grid import (AXIS, COMPS, E_COMPS, PAIRS, Grid, add, apply_op, d_e_to_h, d_h_to_e,
                   line_operator_coeffs, material_at_samples, scale, solve_implicit, solve_lines,
                   solve_lines4)


@dataclass
class Source:
    comp: str                     # "ex", "ey" or "ez"
    k: int
    j: int
    i: int
    current: Callable[[float], float]


@dataclass
class Problem:
    grid: Grid
    dt: float
    eps_r_cell: np.ndarray | None = None
    mu_r_cell: np.ndarray | None = None
    source: Source | None = None
    sigma_cell: np.ndarray | None = None     # electric conductivity [S/m] per cell (lossy media)
    mat: dict = field(init=False)

    def __post_init__(self):
        self.mat = material_at_samples(self.grid, self.eps_r_cell, self.mu_r_cell, self.sigma_cell)

    def f(self, t: float) -> dict | None:
        """Source vector f = (-J/eps, 0) at time t, or None."""
        if self.source is None:
            return None
        s = self.source
        g = self.grid
        area = {"ex": g.dy * g.dz, "ey": g.dx * g.dz, "ez": g.dx * g.dy}[s.comp]
        v = g.zeros()
        v[s.comp][s.k, s.j, s.i] = -float(s.current(t)) / (area * self.mat[s.comp][s.k, s.j, s.i])
        return v


def _plus(u, v, alpha):
    return u if v is None else add(u, v, alpha)


# ---------------------------------------------------------------------------
# Original schemes (Sec. II)
# ---------------------------------------------------------------------------

def _cn_substep(P: Problem, u: dict, op_implicit: str, op_explicit: str, tau: float, f) -> dict:
    """(I - tau*O_i) u' = (I + tau*O_e) u + tau*f."""
    rhs = add(u, apply_op(P.grid, P.mat, op_explicit, u), tau)
    rhs = _plus(rhs, f, tau)
    return solve_implicit(P.grid, P.mat, op_implicit, tau, rhs)


def orig_adi_step(P: Problem, u: dict, n: int) -> dict:
    """Peaceman-Rachford ADI, Eq. 1 (1a then 1b)."""
    tau = P.dt / 2
    f = P.f((n + 0.5) * P.dt)
    uh = _cn_substep(P, u, "A", "B", tau, f)
    return _cn_substep(P, uh, "B", "A", tau, f)


def orig_lod1_step(P: Problem, u: dict, n: int, return_half: bool = False):
    """LOD1 / SS1, Eq. 11 (11a then 11b)."""
    tau = P.dt / 2
    f = P.f((n + 0.5) * P.dt)
    uh = _cn_substep(P, u, "A", "A", tau, f)
    u1 = _cn_substep(P, uh, "B", "B", tau, f)
    return (u1, uh) if return_half else u1


def orig_ss2_step(P: Problem, u: dict, n: int) -> dict:
    """Strang split-step SS2, Eq. 16 (three Crank-Nicolson sub-steps)."""
    f = P.f((n + 0.5) * P.dt)
    u1 = _cn_substep(P, u, "A", "A", P.dt / 4, f)
    u2 = _cn_substep(P, u1, "B", "B", P.dt / 2, f)
    return _cn_substep(P, u2, "A", "A", P.dt / 4, f)


def orig_lod2_input(P: Problem, u0: dict, n0: int = 0) -> dict:
    """LOD2 input processing, Eq. 19: (I - dt/4 B) u^{n0+1/4} = (I + dt/4 B) u^{n0}
    (+ (dt/4) f(t_{n0} + dt/2))."""
    return _cn_substep(P, u0, "B", "B", P.dt / 4, P.f((n0 + 0.5) * P.dt))


def orig_lod2_step(P: Problem, u: dict, n: int) -> dict:
    """LOD2 main loop, Eq. 18 (the LOD1 step of Eq. 11): the A sub-step takes
    f(t_n + dt/2), the B sub-step (centred on t_{n+1}) the mean of f(t_n + dt/2)
    and f(t_n + 3dt/2)."""
    tau = P.dt / 2
    fa = P.f((n + 0.5) * P.dt)
    fb = _mean_f(P, n)
    uh = _cn_substep(P, u, "A", "A", tau, fa)
    return _cn_substep(P, uh, "B", "B", tau, fb)


def orig_lod2_output(P: Problem, u: dict, n_next: int = 0) -> dict:
    """LOD2 output processing, Eq. 20: (I + dt/4 B) u^{n+1} = (I - dt/4 B) u^{n+5/4}
    (- (dt/4) f(t_{n+1} + dt/2)); ``n_next`` = n + 1."""
    return _cn_substep(P, u, "B", "B", -P.dt / 4, P.f((n_next + 0.5) * P.dt))


def _mean_f(P: Problem, n: int):
    """(f(t_n + dt/2) + f(t_n + 3dt/2)) / 2, or None without a source."""
    fa = P.f((n + 0.5) * P.dt)
    if fa is None:
        return None
    return scale(add(fa, P.f((n + 1.5) * P.dt)), 0.5)


def run_original(P: Problem, scheme: str, u0: dict, steps: int) -> dict:
    u = {c: u0[c].copy() for c in COMPS}
    if scheme == "adi":
        for n in range(steps):
            u = orig_adi_step(P, u, n)
    elif scheme == "lod1":
        for n in range(steps):
            u = orig_lod1_step(P, u, n)
    elif scheme == "ss2":
        for n in range(steps):
            u = orig_ss2_step(P, u, n)
    elif scheme == "lod2":
        u = orig_lod2_input(P, u)
        for n in range(steps):
            u = orig_lod2_step(P, u, n)
        u = orig_lod2_output(P, u, steps)
    else:
        raise ValueError(scheme)
    return u


# ---------------------------------------------------------------------------
# The fundamental updating procedure (Sec. III)
# ---------------------------------------------------------------------------

def procedure(P: Problem, state: dict, op: str, h: float, rhs_src: dict | None = None,
              post_src: dict | None = None):
    """One updating procedure of a fundamental scheme, (1/2 I - h/4 O) w = state
    followed by state <- w - state, in the per-component form of Sec. III:

      implicit  1/2 w - (b/2) d(d dw) = E + sgn * b * d(H)      (Eqs. 38, 41, 45, 48)
      explicit  H <- H + sgn * d * d(w)                        (Eqs. 43-44, 51-52)
      subtract  E <- w - E                                     (Eqs. 40, 47, 50)

    with b = h/(2 eps), d = h/(2 mu) (Eq. 36), sgn = +1 for A and -1 for B.
    In a lossy medium the implicit diagonal is 1/2 + b sigma / 4 (the
    operator's half of the loss).
    ``rhs_src`` is added to the implicit right-hand side, ``post_src`` to the
    new E state.  Returns (new_state, w, H_before)."""
    g = P.grid
    new = {}
    w_all = {}
    for ec, hc, ax, sgn in PAIRS[op]:
        a = AXIS[ax]
        sp = g.spacing[ax]
        mask = g.e_interior_mask(ec)
        b = h / (2.0 * P.mat[ec])
        d = h / (2.0 * P.mat[hc])
        r = state[ec] + sgn * b * d_h_to_e(g, state[hc], a, sp, g.shape(ec))
        if rhs_src is not None:
            r = r + rhs_src[ec]
        r = r * mask
        diag = 0.5 + 0.25 * b * P.mat["sigma"][ec] if "sigma" in P.mat else 0.5
        if g.order == 4:
            # 1/2 w - (b/2) D(d D w) with the fourth-order differences
            w = solve_lines4(diag, 0.5 * b, d, r, a, sp) * mask
        else:
            lo, ce, up = line_operator_coeffs(b, d, a, sp)
            # 1/2 w - (b/2) d(d dw): the line operator scaled by 1/2
            w = solve_lines(diag, 0.5 * lo, 0.5 * ce, 0.5 * up, r, a) * mask
        w_all[ec] = w
        new[hc] = state[hc] + sgn * d * d_e_to_h(g, w, a, sp)
        e_new = w - state[ec]
        if post_src is not None:
            e_new = e_new + post_src[ec]
        new[ec] = e_new * mask
    return new, w_all, {c: state[c] for c in ("hx", "hy", "hz")}


# ---------------------------------------------------------------------------
# FADI (Eqs. 7-10, component form Eqs. 37-44)
# ---------------------------------------------------------------------------

def fadi_init(P: Problem, u0: dict) -> dict:
    """Input initialization: v^{-1/2} = (I - dt/2 B) u^0 (Eq. 10), u~^0 = 2u^0
    (Eq. 7), v^0 = u~^0 - v^{-1/2} (Eq. 8a); plus the first sub-step's source."""
    vm = add(u0, apply_op(P.grid, P.mat, "B", u0), -P.dt / 2)
    v0 = add(scale(u0, 2.0), vm, -1.0)
    return _plus(v0, P.f(0.5 * P.dt), P.dt / 2)


def fadi_step(P: Problem, v: dict, n: int, want_output: bool = False):
    """One FADI step v^n -> v^{n+1} (Eqs. 8a-8d in the form of Eqs. 37-44).
    With ``want_output`` also returns u^{n+1} = u~^{n+1}/2 (Eq. 9), where
    E~^{n+1} is the B-solve result and H~^{n+1} = 2 h^{n+1/2} - d dE~ (Eq. 42)."""
    dt = P.dt
    fa = P.f((n + 0.5) * dt)            # source of this step's second sub-step
    fb = P.f((n + 1.5) * dt)            # source of the next step's first sub-step
    vh, _, _ = procedure(P, v, "A", dt, post_src=None if fa is None else scale(fa, dt / 2))
    v1, wB, hB = procedure(P, vh, "B", dt, post_src=None if fb is None else scale(fb, dt / 2))
    if not want_output:
        return v1
    out = {}
    for ec in E_COMPS:
        out[ec] = 0.5 * wB[ec]
    for hc in ("hx", "hy", "hz"):
        # H~ = 2 h^{n+1/2} + sgn d dE~ = h^{n+1/2} + h^{n+1}
        out[hc] = 0.5 * (hB[hc] + v1[hc])
    return v1, out


def fadi_output_from_state(P: Problem, v: dict, n_next: int) -> dict:
    """u^n from the FADI state v^n alone: v^n = (I + dt/2 B) u^n + (dt/2) f,
    so u^n = (I + dt/2 B)^{-1} (v^n - (dt/2) f)  (from Eqs. 2a and 8a);
    ``n_next`` is the index of the step that would come next."""
    f = P.f((n_next + 0.5) * P.dt)
    r = _plus(v, f, -P.dt / 2)
    return solve_implicit(P.grid, P.mat, "B", -P.dt / 2, r)


def run_fadi(P: Problem, u0: dict, steps: int, probes=(), record_state=False):
    """Run FADI for ``steps`` steps from u^0.  Returns (u^steps, v^steps, probe
    series) where probe series[p][n] is the output field at probe p after
    step n+1."""
    v = fadi_init(P, u0)
    series = [np.zeros(steps) for _ in probes]
    u = {c: u0[c].copy() for c in COMPS}
    for n in range(steps):
        v, u = fadi_step(P, v, n, want_output=True)
        for p, (c, i, j, k) in enumerate(probes):
            series[p][n] = u[c][k, j, i]
    return u, v, series


# ---------------------------------------------------------------------------
# FLOD (Eq. 15), FSS (Eq. 17), FLOD2 (Eqs. 21-23)
# ---------------------------------------------------------------------------

def flod_step(P: Problem, u: dict, n: int) -> dict:
    """Eqs. 15a-15d: (1/2 I - dt/4 A) v = u^n, u^{n+1/2} = v - u^n, then B."""
    f = P.f((n + 0.5) * P.dt)
    src = None if f is None else scale(f, P.dt / 4)
    uh, _, _ = procedure(P, u, "A", P.dt, rhs_src=src)
    u1, _, _ = procedure(P, uh, "B", P.dt, rhs_src=src)
    return u1


def fss_step(P: Problem, u: dict, n: int) -> dict:
    """Eqs. 17a-17f: procedures with dt/8 (A), dt/4 (B), dt/8 (A) coefficients,
    i.e. procedure lengths dt/2, dt, dt/2."""
    f = P.f((n + 0.5) * P.dt)
    sa = None if f is None else scale(f, P.dt / 8)
    sb = None if f is None else scale(f, P.dt / 4)
    u1, _, _ = procedure(P, u, "A", P.dt / 2, rhs_src=sa)
    u2, _, _ = procedure(P, u1, "B", P.dt, rhs_src=sb)
    u3, _, _ = procedure(P, u2, "A", P.dt / 2, rhs_src=sa)
    return u3


def flod2_input(P: Problem, u0: dict, n0: int = 0) -> dict:
    """Eq. 22: (1/2 I - dt/8 B) v = u^{n0} (+ (dt/8) f(t_{n0} + dt/2)),
    u^{n0+1/4} = v - u^{n0} (procedure length dt/2)."""
    f = P.f((n0 + 0.5) * P.dt)
    return procedure(P, u0, "B", P.dt / 2, rhs_src=None if f is None else scale(f, P.dt / 8))[0]


def flod2_step(P: Problem, u: dict, n: int) -> dict:
    """Eq. 21: the FLOD procedures with +(dt/4) f in each implicit right-hand
    side, f(t_n + dt/2) for A and the mean of f(t_n + dt/2), f(t_n + 3dt/2)
    for B (the sub-step centred on t_{n+1})."""
    fa = P.f((n + 0.5) * P.dt)
    fb = _mean_f(P, n)
    uh, _, _ = procedure(P, u, "A", P.dt, rhs_src=None if fa is None else scale(fa, P.dt / 4))
    u1, _, _ = procedure(P, uh, "B", P.dt, rhs_src=None if fb is None else scale(fb, P.dt / 4))
    return u1


def flod2_output(P: Problem, u: dict, n_next: int = 0) -> dict:
    """Eq. 23: (1/2 I + dt/8 B) v = u^{n+5/4} (- (dt/8) f(t_{n+1} + dt/2)),
    u^{n+1} = v - u^{n+5/4} (a procedure of length -dt/2); n_next = n + 1."""
    f = P.f((n_next + 0.5) * P.dt)
    return procedure(P, u, "B", -P.dt / 2, rhs_src=None if f is None else scale(f, -P.dt / 8))[0]


def run_fundamental(P: Problem, scheme: str, u0: dict, steps: int, probes=()):
    """Run a fundamental scheme; returns (field u, scheme state, probe series)."""
    if scheme == "fadi":
        return run_fadi(P, u0, steps, probes)
    u = {c: u0[c].copy() for c in COMPS}
    series = [np.zeros(steps) for _ in probes]
    if scheme == "flod2":
        u = flod2_input(P, u)
    for n in range(steps):
        if scheme == "flod":
            u = flod_step(P, u, n)
        elif scheme == "flod2":
            u = flod2_step(P, u, n)
        elif scheme == "fss":
            u = fss_step(P, u, n)
        else:
            raise ValueError(scheme)
        out = flod2_output(P, u, n + 1) if (scheme == "flod2" and probes) else u
        for p, (c, i, j, k) in enumerate(probes):
            series[p][n] = out[c][k, j, i]
    field_out = flod2_output(P, u, steps) if scheme == "flod2" else u
    return field_out, u, series


# ---------------------------------------------------------------------------
# D'Yakonov (Beam-Warming) and Douglas-Gunn splittings (Sec. II, "Fundamental
# Implications and Significance"): extra equivalence pins of the procedure
# ---------------------------------------------------------------------------

def orig_dy_step(P: Problem, u: dict) -> dict:
    """Eq. 25: (I - dt/2 A) u* = (I + dt/2 A)(I + dt/2 B) u^n, (I - dt/2 B) u^{n+1} = u*."""
    tau = P.dt / 2
    w = add(u, apply_op(P.grid, P.mat, "B", u), tau)
    rhs = add(w, apply_op(P.grid, P.mat, "A", w), tau)
    ustar = solve_implicit(P.grid, P.mat, "A", tau, rhs)
    return solve_implicit(P.grid, P.mat, "B", tau, ustar)


def fast_dy_init(P: Problem, u0: dict) -> dict:
    """Eq. 27: v^{-1/2} = (1/2 I - dt/4 B) u^0."""
    return add(scale(u0, 0.5), apply_op(P.grid, P.mat, "B", u0), -P.dt / 4)


def fast_dy_step(P: Problem, u: dict, vm: dict):
    """Eq. 26 from (u^n, v^{n-1/2}): v^n = u^n - v^{n-1/2}; (1/2 I - dt/4 A) u^{n+1/2} = v^n;
    v^{n+1/2} = u^{n+1/2} - v^n; (1/2 I - dt/4 B) u^{n+1} = v^{n+1/2}.  The two solve +
    subtract pairs are the updating procedure.  Returns (u^{n+1}, v^{n+1/2})."""
    v = add(u, vm, -1.0)
    vh, _, _ = procedure(P, v, "A", P.dt)          # state <- u^{n+1/2} - v^n = v^{n+1/2}
    v1, _, _ = procedure(P, vh, "B", P.dt)         # state <- u^{n+1} - v^{n+1/2}
    return add(v1, vh), vh


def orig_dg_step(P: Problem, u: dict):
    """Eq. 29 (delta formulation): (I - dt/2 A) du* = dt (A + B) u^n,
    (I - dt/2 B) du = du*, u^{n+1} = u^n + du.  Returns (u^{n+1}, du*, du)."""
    tau = P.dt / 2
    rhs = scale(add(apply_op(P.grid, P.mat, "A", u), apply_op(P.grid, P.mat, "B", u)), P.dt)
    dus = solve_implicit(P.grid, P.mat, "A", tau, rhs)
    du = solve_implicit(P.grid, P.mat, "B", tau, dus)
    return add(u, du), dus, du
