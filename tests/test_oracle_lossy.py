"""Pins for lossy (conductive) media in the oracle.

The paper writes A and B for a lossless medium (Sec. III, Eqs. 33-34) but
states its splitting formulae (Sec. II) for generic linear operators.  The
reading: an electric conductivity sigma adds -sigma/eps E to dE/dt, split
evenly between A and B on the E rows; a procedure of length h then has the
implicit diagonal 1/2 + b sigma / 4.  Pinned here against:

* dense brute force (A and B assembled entry by entry with the loss
  diagonal) for the original schemes, with and without a source;
* the paper's central claim, fundamental = original, with loss;
* the physics of the loss: the symmetric part of A + B in the energy
  product is exactly -diag(sigma dV) on the E unknowns (Joule heating), so
  the field energy of every scheme decreases monotonically at any CFL;
* the closed form of a damped cavity mode: the 6 x 6 operator has the
  eigenvalues -sigma/(2 eps) +- i sqrt(c^2 k'^2 - (sigma/(2 eps))^2) and
  -sigma/eps (static E) and 0 (static H); the modal evolution equals the
  stepper;
* convergence of a sourced lossy run to the semi-discrete system (RK4) at
  the orders of Table I.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import dense as D
from oracle import grid as G
from oracle import invariants as I
from oracle import modal as M
from oracle import schemes as S
from oracle import semidiscrete as SD

from test_oracle_schemes import random_state, rel


def lossy_problem(seed, nx=4, ny=5, nz=3, cfl=4.0, source=False, sigma_max=2.0):
    rng = np.random.default_rng(seed)
    g = G.Grid(nx, ny, nz, 1.0e-3, 1.3e-3, 0.8e-3)
    eps = rng.uniform(1, 6, (nz, ny, nx))
    mu = rng.uniform(1, 2, (nz, ny, nx))
    sig = rng.uniform(0, sigma_max, (nz, ny, nx))
    src = S.Source("ez", nz // 2, ny // 2, nx // 2, lambda t: np.sin(2e10 * t) + 0.3) if source else None
    P = S.Problem(g, cfl * g.dt_cfl(), eps, mu, src, sigma_cell=sig)
    return P, random_state(g, rng)


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("scheme", ["adi", "lod1", "ss2"])
def test_lossy_structured_original_matches_dense(scheme, source):
    P, u0 = lossy_problem(11, source=source)
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


@pytest.mark.parametrize("source", [False, True])
@pytest.mark.parametrize("orig,fund", [("adi", "fadi"), ("lod1", "flod"), ("ss2", "fss"), ("lod2", "flod2")])
def test_lossy_fundamental_equals_original(orig, fund, source):
    P, u0 = lossy_problem(21, nx=6, ny=5, nz=7, cfl=6.0, source=source)
    uo = S.run_original(P, orig, u0, 12)
    uf, _, _ = S.run_fundamental(P, fund, u0, 12)
    assert rel(uf, uo) < 1e-12


def test_loss_is_the_symmetric_part_in_the_energy_product():
    """W (A + B) + (A + B)^T W = -2 diag(sigma) on the E unknowns and 0
    elsewhere (W = diag(eps, mu)): the Joule loss dW/dt = -dV sum sigma E^2."""
    P, _ = lossy_problem(12)
    g = P.grid
    A, B = D.assemble(g, P.mat)
    wdiag = D.to_vec(g, {c: P.mat[c] for c in G.COMPS})
    mask = D.to_vec(g, {c: (g.e_interior_mask(c) if c in G.E_COMPS else np.ones(g.shape(c))) for c in G.COMPS})
    keep = mask > 0
    sig = D.to_vec(g, {c: (P.mat["sigma"][c] if c in G.E_COMPS else np.zeros(g.shape(c))) for c in G.COMPS})
    S_ = (np.diag(wdiag) @ (A + B))[np.ix_(keep, keep)]
    sym = S_ + S_.T
    expect = np.diag(-2.0 * sig[keep])
    assert np.max(np.abs(sym - expect)) < 1e-12 * np.max(np.abs(S_))
    assert np.max(sig) > 0


@pytest.mark.parametrize("cfl", [4.0, 10.0])
@pytest.mark.parametrize("scheme", ["flod", "fss", "fadi"])
def test_lossy_energy_decreases_every_step(scheme, cfl):
    """Each procedure is the Cayley transform of a dissipative operator: the
    invariant (W(u) for FLOD/FSS, W(v) for FADI) never grows, and it falls."""
    P, u0 = lossy_problem(50, nx=7, ny=6, nz=5, cfl=cfl)
    g = P.grid
    x = S.fadi_init(P, u0) if scheme == "fadi" else u0
    step = {"fadi": S.fadi_step, "flod": S.flod_step, "fss": S.fss_step}[scheme]
    e = [I.energy(g, P.mat, x)]
    for n in range(30):
        x = step(P, x, n)
        e.append(I.energy(g, P.mat, x))
    assert all(b <= a * (1 + 1e-14) for a, b in zip(e, e[1:]))
    assert e[-1] < 0.9 * e[0]


def test_damped_cavity_mode_eigenvalues_closed_form():
    """Homogeneous eps, sigma: the mode's 6 x 6 operator A + B has the damped
    oscillator's eigenvalues (a double pair), -sigma/eps for the static E
    component and 0 for the static H component."""
    g = G.Grid(9, 8, 7, 1e-3, 1.1e-3, 0.9e-3)
    eps = 3.0 * G.EPS0
    sigma = 0.4
    m, n, p = 2, 3, 4
    A, B = M.mode_operators(g, m, n, p, eps=eps, sigma=sigma)
    lam = np.linalg.eigvals(A + B)
    kp2 = sum(((2.0 / d) * math.sin(k * math.pi / N / 2.0)) ** 2
              for k, d, N in ((m, g.dx, g.nx), (n, g.dy, g.ny), (p, g.dz, g.nz)))
    a = sigma / (2 * eps)
    wd = math.sqrt(kp2 / (eps * G.MU0) - a * a)
    expect = [-a - 1j * wd, -a - 1j * wd, -a + 1j * wd, -a + 1j * wd, -2 * a + 0j, 0j]
    left = list(lam)
    for e in expect:                  # match as multisets (roundoff splits the double pair)
        q = int(np.argmin([abs(x - e) for x in left]))
        assert abs(left.pop(q) - e) < 1e-9 * wd, (lam, expect)


@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss"])
def test_lossy_modal_evolution_equals_stepper(scheme):
    nx, ny, nz = 10, 8, 6
    d = (1e-3, 1.2e-3, 0.9e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 6.0 * g.dt_cfl()
    eps_r, sigma = 2.5, 0.3
    modes = W.random_modes(3, nx, ny, nz, *d, count=3, mmax=5)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    steps = 25
    P = S.Problem(g, dt, eps_r_cell=np.full((nz, ny, nx), eps_r), sigma_cell=np.full((nz, ny, nx), sigma))
    ref, _, _ = S.run_fundamental(P, scheme, u0, steps)
    got = M.field_after(g, dt, scheme, modes, steps, eps_r=eps_r, sigma=sigma)
    assert rel(got, ref) < 1e-12
    # and the field has decayed as the loss says it should (about exp(-sigma t / (2 eps)))
    assert I.energy(g, P.mat, ref) < 0.8 * I.energy(g, P.mat, u0)


def test_rk4_lossy_mode_matches_the_closed_form():
    """The semi-discrete reference in a lossy medium: RK4 on a damped mode
    against exp(t (A + B)) of its 6 x 6 operator."""
    g = G.Grid(8, 7, 6, 1e-3, 1e-3, 1e-3)
    eps_r, sigma = 2.0, 0.5
    P = S.Problem(g, 1.0, eps_r_cell=np.full((6, 7, 8), eps_r), sigma_cell=np.full((6, 7, 8), sigma))
    c0 = np.array([0.3, -0.5, 0.7, 1e-3, -2e-3, 5e-4])
    u0 = M.fields_from_modes(g, [(2, 3, 1, c0)])
    t_end = 40 * g.dt_cfl()
    A, B = M.mode_operators(g, 2, 3, 1, eps=G.EPS0 * eps_r, sigma=sigma)
    exact = M.fields_from_modes(g, [(2, 3, 1, scipy.linalg.expm(t_end * (A + B)) @ c0)])
    u = SD.rk4(g, P.mat, None, u0, t_end, SD.rk4_stable_steps(g, t_end, 0.025))
    assert rel(u, exact) < 2e-7


@pytest.mark.parametrize("scheme,order", [("fadi", 2.0), ("flod", 1.0), ("fss", 2.0), ("flod2", 2.0)])
def test_lossy_sourced_run_converges_to_the_semi_discrete_system(scheme, order):
    nx, ny, nz = 6, 5, 7
    g = G.Grid(nx, ny, nz, 1e-3, 1.2e-3, 0.9e-3)
    rng = np.random.default_rng(7)
    eps = rng.uniform(1, 4, (nz, ny, nx))
    sig = rng.uniform(0.0, 1.0, (nz, ny, nx))
    f0, sg, t0 = 15e9, 25e-12, 60e-12
    src = S.Source("ez", 3, 2, 3, lambda t: math.exp(-((t - t0) / sg) ** 2) * math.sin(2 * math.pi * f0 * (t - t0)))
    T = 160e-12
    mat = S.Problem(g, 1.0, eps_r_cell=eps, sigma_cell=sig).mat
    ref = SD.rk4(g, mat, src, g.zeros(), T, SD.rk4_stable_steps(g, T, 0.05))
    steps = {"fadi": (80, 160, 320), "flod": (640, 1280, 2560), "fss": (160, 320, 640), "flod2": (80, 160, 320)}[scheme]
    errs = []
    for n in steps:
        P = S.Problem(g, T / n, eps_r_cell=eps, source=src, sigma_cell=sig)
        u, _, _ = S.run_fundamental(P, scheme, g.zeros(), n)
        errs.append(rel(u, ref))
    p = math.log2(errs[-2] / errs[-1])
    assert p == pytest.approx(order, abs=0.15), errs
