"""Pins for the oracle's schemes.

* Structured operators and original schemes vs dense brute force assembled
  entry by entry from Eqs. 33-34 (tiny grids, uneven spacings, eps and mu
  varying per cell, with and without a source).
* The paper's central claim: fundamental forms give the original schemes'
  fields up to roundoff (Sec. II: Eqs. 8-10 vs 1, 15 vs 11, 17 vs 16,
  21-23 vs 18-20).
* The LOD-ADI link of Sec. II-E (Eq. 24).
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import grid as G
from oracle import schemes as S


def rel(a: dict, b: dict) -> float:
    num = sum(float(np.sum((a[c] - b[c]) ** 2)) for c in G.COMPS)
    den = sum(float(np.sum(b[c] ** 2)) for c in G.COMPS)
    return (num / den) ** 0.5


def random_state(g, rng):
    u = {}
    for c in G.COMPS:
        u[c] = rng.standard_normal(g.shape(c))
    for c in G.E_COMPS:
        u[c] *= g.e_interior_mask(c)
    # scale H to the same energy scale as E
    for c in G.H_COMPS:
        u[c] /= 376.73
    return u


def make_problem(seed, nx=3, ny=4, nz=5, cfl=4.0, inhom=True, source=False):
    rng = np.random.default_rng(seed)
    g = G.Grid(nx, ny, nz, 1.0e-3, 1.3e-3, 0.8e-3)
    eps = rng.uniform(1, 6, (nz, ny, nx)) if inhom else None
    mu = rng.uniform(1, 2, (nz, ny, nx)) if inhom else None
    src = None
    if source:
        src = S.Source("ez", nz // 2, ny // 2, nx // 2, lambda t: np.sin(2e10 * t) + 0.3)
    P = S.Problem(g, cfl * g.dt_cfl(), eps, mu, src)
    return P, random_state(g, rng)


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("scheme", ["adi", "lod1", "ss2"])
def test_structured_original_matches_dense(scheme, source):
    P, u0 = make_problem(11, source=source)
    g = P.grid
    A, B = D.assemble(g, P.mat)
    x = D.to_vec(g, u0)
    u = u0
    step_dense = {"adi": D.adi_step, "lod1": D.lod1_step, "ss2": D.ss2_step}[scheme]
    step = {"adi": S.orig_adi_step, "lod1": S.orig_lod1_step, "ss2": S.orig_ss2_step}[scheme]
    for n in range(4):
        f = P.f((n + 0.5) * P.dt)
        x = step_dense(A, B, P.dt, x, None if f is None else D.to_vec(g, f))
        u = step(P, u, n)
    assert rel(u, D.from_vec(g, x)) < 1e-13


def test_dense_operators_are_skew_in_energy_product():
    """<Au, w>_W = -<u, Aw>_W (and for B): the property behind unconditional
    stability; W = diag(eps at E samples, mu at H samples)."""
    P, _ = make_problem(12)
    g = P.grid
    A, B = D.assemble(g, P.mat)
    wdiag = D.to_vec(g, {c: P.mat[c] for c in G.COMPS})
    mask = D.to_vec(g, {c: (g.e_interior_mask(c) if c in G.E_COMPS else np.ones(g.shape(c)))
                        for c in G.COMPS})
    keep = mask > 0            # the unknowns: wall E samples are fixed at 0
    Wm = np.diag(wdiag)
    for O in (A, B):
        S_ = (Wm @ O)[np.ix_(keep, keep)]
        assert np.max(np.abs(S_ + S_.T)) < 1e-12 * np.max(np.abs(S_))


def test_split_operators_sum_to_curl():
    """A + B applied to a field equals the Yee curl update (1/eps curl H, -1/mu curl E)."""
    P, u = make_problem(13, inhom=False)
    g = P.grid
    Au = G.apply_op(g, P.mat, "A", u)
    Bu = G.apply_op(g, P.mat, "B", u)
    # curl H . x at Ex: dHz/dy - dHy/dz
    dhz = G.diff_h_to_e(u["hz"], 1, g.dy, g.shape("ex"))
    dhy = G.diff_h_to_e(u["hy"], 0, g.dz, g.shape("ex"))
    ref = (dhz - dhy) / P.mat["ex"] * g.e_interior_mask("ex")
    assert np.allclose(Au["ex"] + Bu["ex"], ref, rtol=1e-14, atol=0)
    # -(curl E) . z at Hz: -(dEy/dx - dEx/dy)
    ref = -(G.diff_e_to_h(u["ey"], 2, g.dx) - G.diff_e_to_h(u["ex"], 1, g.dy)) / P.mat["hz"]
    assert np.allclose(Au["hz"] + Bu["hz"], ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("orig,fund", [("adi", "fadi"), ("lod1", "flod"), ("ss2", "fss"), ("lod2", "flod2")])
def test_fundamental_equals_original(orig, fund, source):
    P, u0 = make_problem(21, nx=6, ny=5, nz=7, cfl=6.0, source=source)
    uo = S.run_original(P, orig, u0, 12)
    uf, _, _ = S.run_fundamental(P, fund, u0, 12)
    assert rel(uf, uo) < 1e-12


def test_fadi_2d_gaussian_equals_original_adi():
    """The 2-D TM case (nz = 1): Gaussian Ez pulse, CFL 5, vs the original ADI."""
    f, _ = W.gaussian_ez_2d(24, 20, 3.0, seed=1)
    g = G.Grid(24, 20, 1, 1e-3, 1e-3, 1e-3)
    P = S.Problem(g, 5 * g.dt_cfl())
    uo = S.run_original(P, "adi", f, 30)
    uf, _, _ = S.run_fundamental(P, "fadi", f, 30)
    assert rel(uf, uo) < 1e-12
    # TM: Ex, Ey, Hz stay exactly zero
    for c in ("ex", "ey", "hz"):
        assert np.max(np.abs(uf[c])) == 0.0


def test_fadi_output_from_state_matches_eq9():
    P, u0 = make_problem(31, source=True)
    v = S.fadi_init(P, u0)
    for n in range(6):
        v, u = S.fadi_step(P, v, n, want_output=True)
    us = S.fadi_output_from_state(P, v, 6)
    assert rel(us, u) < 1e-12


def test_fadi_init_is_exact():
    """Eq. 10 initialization loses nothing: the field output of the initial
    state (before any step) is u^0 itself."""
    P, u0 = make_problem(32)
    v0 = S.fadi_init(P, u0)
    assert rel(S.fadi_output_from_state(P, v0, 0), u0) < 1e-13


def test_lod_adi_link():
    """Sec. II-E (Eq. 24): starting LOD1 from u^0_LOD = (1/2 I + dt/4 B)(2 u^0),
    the LOD auxiliary v^{n+1} = u^{n+1} + u^{n+1/2} equals 2 u^{n+1} of ADI."""
    P, u0 = make_problem(41, nx=5, ny=6, nz=4, cfl=3.0)
    g = P.grid
    ulod = G.add(u0, G.apply_op(g, P.mat, "B", u0), P.dt / 2)
    uadi = {c: u0[c].copy() for c in G.COMPS}
    for n in range(8):
        ulod, uhalf = S.orig_lod1_step(P, ulod, n, return_half=True)
        uadi = S.orig_adi_step(P, uadi, n)
        vlod = G.add(ulod, uhalf)
        assert rel(vlod, G.scale(uadi, 2.0)) < 1e-12


def test_material_averaging_by_hand():
    """Edge/face averaging reading: one cell of eps_r = 5 in a 2x2x2 grid."""
    g = G.Grid(2, 2, 2, 1, 1, 1)
    er = np.ones((2, 2, 2))
    er[1, 1, 1] = 5.0            # cell (i=1, j=1, k=1)
    mr = np.ones((2, 2, 2))
    mr[0, 0, 0] = 3.0
    m = G.material_at_samples(g, er, mr)
    e = m["ex"] / G.EPS0
    # Ex edge (i+1/2=1.5, j=1, k=1) touches cells (1, 0..1, 0..1): one of four is 5
    assert e[1, 1, 1] == pytest.approx(2.0)
    # Ex edge on the wall corner (1.5, 2, 2): only cell (1,1,1) -> 5
    assert e[2, 2, 1] == pytest.approx(5.0)
    # Ex edge (0.5, 1, 1): cells (0, .., ..) all 1
    assert e[1, 1, 0] == pytest.approx(1.0)
    h = m["hx"] / G.MU0
    # Hx face (i=1, j+1/2=0.5, k+1/2=0.5) between cells (0,0,0) and (1,0,0)
    assert h[0, 0, 1] == pytest.approx(2.0)
    assert h[0, 0, 0] == pytest.approx(3.0)     # wall face: one cell only
    assert m["hz"][0, 0, 0] / G.MU0 == pytest.approx(3.0)
    assert m["hy"][0, 1, 0] / G.MU0 == pytest.approx(2.0)
