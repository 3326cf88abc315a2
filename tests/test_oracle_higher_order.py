"""Pins for the fourth-order difference operators of the oracle.

The paper names higher-order difference operators as a variant of its
schemes (end of Sec. III-A) without formulae; the reading: every first
difference of A and B (Eqs. 33-34) becomes the fourth-order staggered
central difference (9/8, -1/24), with PEC images past the walls (tangential
E odd, H even).  Pinned against:

* the difference itself: fourth-order accurate on smooth data, and its
  symbol on cavity-mode samples is (2/d)(9/8 sin(kd/2) - 1/24 sin(3kd/2));
* skewness: the two differences are exact negative transposes, so dense
  A and B (assembled entry by entry, independently of the structured code)
  are skew in the energy product;
* dense brute force for the original schemes, fundamental = original for
  all four schemes, exact energy conservation at large CFL numbers;
* the closed-form cavity modes and the dispersion relation with the
  fourth-order symbol, against the stepper.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import grid as G
from oracle import invariants as I
from oracle import modal as M
from oracle import schemes as S

from test_oracle_schemes import random_state, rel


def problem4(seed, nx=5, ny=6, nz=4, cfl=4.0, inhom=True, source=False):
    rng = np.random.default_rng(seed)
    g = G.Grid(nx, ny, nz, 1.0e-3, 1.3e-3, 0.8e-3, order=4)
    eps = rng.uniform(1, 6, (nz, ny, nx)) if inhom else None
    mu = rng.uniform(1, 2, (nz, ny, nx)) if inhom else None
    src = S.Source("ez", nz // 2, ny // 2, nx // 2, lambda t: np.sin(2e10 * t) + 0.3) if source else None
    P = S.Problem(g, cfl * g.dt_cfl(), eps, mu, src)
    return P, random_state(g, rng)


def test_fourth_order_difference_converges_at_fourth_order():
    """d/dx of sin(2 pi x) sampled on staggered points of [0, 1] (an odd
    function about both walls, as tangential E), against 2 pi cos: the
    maximum error falls 16-fold per halving of d."""
    errs = []
    for n in (16, 32, 64):
        d = 1.0 / n
        x = np.arange(n + 1) * d
        e = np.sin(2 * math.pi * x)
        got = G.diff_e_to_h4(e, 0, d)
        exact = 2 * math.pi * np.cos(2 * math.pi * (np.arange(n) + 0.5) * d)
        errs.append(np.max(np.abs(got - exact)))
    assert errs[0] / errs[1] == pytest.approx(16.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(16.0, rel=0.05)


@pytest.mark.parametrize("n,m", [(8, 3), (11, 5), (6, 1)])
def test_symbol_on_cavity_mode_samples(n, m):
    """On sin samples (nodes, odd images) and cos samples (faces, even
    images) of a cavity mode the difference acts as the closed-form symbol,
    images included: the modes stay exact eigenfunctions."""
    d = 0.7e-3
    th = m * math.pi / n
    kap = (2 / d) * (9 / 8 * math.sin(th / 2) - 1 / 24 * math.sin(1.5 * th))
    e = np.sin(th * np.arange(n + 1))
    h = np.cos(th * (np.arange(n) + 0.5))
    assert np.allclose(G.diff_e_to_h4(e, 0, d), kap * h, rtol=0, atol=1e-9 * kap)
    assert np.allclose(G.diff_h_to_e4(h, 0, d, (n + 1,))[1:-1], -kap * e[1:-1], rtol=0, atol=1e-9 * kap)
    assert kap == pytest.approx(M.kappa(4, th, d))


@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_differences_are_negative_transposes(n):
    DEH, DHE = G.line_matrices4(n, 0.9e-3)
    assert np.max(np.abs(DHE + DEH.T)) < 1e-9 * np.max(np.abs(DEH))


def test_dense_fourth_order_operators_are_skew_in_energy_product():
    P, _ = problem4(12)
    g = P.grid
    A, B = D.assemble4(g, P.mat)
    wdiag = D.to_vec(g, {c: P.mat[c] for c in G.COMPS})
    mask = D.to_vec(g, {c: (g.e_interior_mask(c) if c in G.E_COMPS else np.ones(g.shape(c))) for c in G.COMPS})
    keep = mask > 0
    for O in (A, B):
        S_ = (np.diag(wdiag) @ O)[np.ix_(keep, keep)]
        assert np.max(np.abs(S_ + S_.T)) < 1e-12 * np.max(np.abs(S_))


def test_structured_fourth_order_operators_match_dense():
    P, u = problem4(13)
    g = P.grid
    A, B = D.assemble4(g, P.mat)
    x = D.to_vec(g, u)
    for op, O in (("A", A), ("B", B)):
        got = D.to_vec(g, G.apply_op(g, P.mat, op, u))
        assert np.max(np.abs(got - O @ x)) < 1e-12 * np.max(np.abs(O @ x))


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("scheme", ["adi", "lod1", "ss2"])
def test_fourth_order_original_matches_dense(scheme, source):
    P, u0 = problem4(11, source=source)
    g = P.grid
    A, B = D.assemble4(g, P.mat)
    x = D.to_vec(g, u0)
    u = u0
    step_dense = {"adi": D.adi_step, "lod1": D.lod1_step, "ss2": D.ss2_step}[scheme]
    step = {"adi": S.orig_adi_step, "lod1": S.orig_lod1_step, "ss2": S.orig_ss2_step}[scheme]
    for n in range(4):
        f = P.f((n + 0.5) * P.dt)
        x = step_dense(A, B, P.dt, x, None if f is None else D.to_vec(g, f))
        u = step(P, u, n)
    assert rel(u, D.from_vec(g, x)) < 1e-13


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("orig,fund", [("adi", "fadi"), ("lod1", "flod"), ("ss2", "fss"), ("lod2", "flod2")])
def test_fourth_order_fundamental_equals_original(orig, fund, source):
    P, u0 = problem4(21, nx=7, ny=5, nz=6, cfl=6.0, source=source)
    uo = S.run_original(P, orig, u0, 10)
    uf, _, _ = S.run_fundamental(P, fund, u0, 10)
    assert rel(uf, uo) < 1e-12


@pytest.mark.parametrize("scheme", ["flod", "fss", "fadi"])
def test_fourth_order_energy_conserved_at_large_cfl(scheme):
    P, u0 = problem4(50, nx=7, ny=6, nz=5, cfl=8.0)
    g = P.grid
    x = S.fadi_init(P, u0) if scheme == "fadi" else u0
    step = {"fadi": S.fadi_step, "flod": S.flod_step, "fss": S.fss_step}[scheme]
    e0 = I.energy(g, P.mat, x)
    for n in range(30):
        x = step(P, x, n)
    assert abs(I.energy(g, P.mat, x) / e0 - 1) < 1e-12


@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss"])
def test_fourth_order_modal_evolution_equals_stepper(scheme):
    nx, ny, nz = 9, 8, 7
    d = (1e-3, 1.2e-3, 0.9e-3)
    g = G.Grid(nx, ny, nz, *d, order=4)
    dt = 6.0 * g.dt_cfl()
    modes = W.random_modes(3, nx, ny, nz, *d, count=3, mmax=4)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    steps = 20
    ref, _, _ = S.run_fundamental(S.Problem(g, dt), scheme, u0, steps)
    got = M.field_after(g, dt, scheme, modes, steps)
    assert rel(got, ref) < 1e-12


def test_fourth_order_cavity_frequency_matches_dispersion_closed_form():
    """A single cavity mode stepped by FADI with fourth-order differences:
    the fitted cos(w dt) equals the ADI dispersion closed form with the
    fourth-order symbol."""
    nx, ny, nz = 10, 9, 8
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d, order=4)
    P = S.Problem(g, 4.0 * g.dt_cfl())
    m, n, p = 2, 3, 1
    md = W.Mode(m, n, p, 1.0, (0.0, 0.0, 1.0))
    # a polarisation orthogonal to the fourth-order symbol vector
    kv = np.array([M.kappa(4, m * math.pi / nx, d), M.kappa(4, n * math.pi / ny, d), M.kappa(4, p * math.pi / nz, d)])
    pol = np.cross(kv, [1.0, 0.0, 0.0])
    md = W.Mode(m, n, p, 1.0, tuple(pol / np.linalg.norm(pol)))
    u0 = W.mode_sum_fields([md], nx, ny, nz)
    shape = {c: W.mode_e_shape(md, nx, ny, nz, unit_amp=True)[c] for c in G.E_COMPS}
    v = S.fadi_init(P, u0)
    series = [I.project(u0, shape)]
    for k in range(40):
        v, u = S.fadi_step(P, v, k, want_output=True)
        series.append(I.project(u, shape))
    c_fit = I.fit_cos_omega_dt(np.array(series))
    w = I.adi_omega(P.dt, m * math.pi / (nx * d), n * math.pi / (ny * d), p * math.pi / (nz * d), d, d, d, order=4)
    assert c_fit == pytest.approx(math.cos(w * P.dt), abs=1e-9)
