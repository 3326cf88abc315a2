"""Further equivalence pins of the oracle (Sec. II, Eqs. 25-30): the D'Yakonov
(Beam-Warming) splitting and the Douglas-Gunn delta formulation step exactly
like Peaceman-Rachford ADI, and their fundamental forms are the FADI iteration."""
import numpy as np
import pytest

from oracle import grid as G
from oracle import schemes as S

from gpu_helpers import energy_norm_rel, random_fields


def problem(seed=3):
    nx, ny, nz = 7, 6, 5
    g = G.Grid(nx, ny, nz, 1e-3, 0.9e-3, 1.1e-3)
    eps = np.random.default_rng(seed).uniform(1.0, 5.0, (nz, ny, nx))
    return S.Problem(g, 6.0 * g.dt_cfl(), eps_r_cell=eps), random_fields(nx, ny, nz, seed=seed + 1)


def test_dyakonov_steps_like_adi():
    """(I - tA)^{-1} commutes with (I + tA): Eq. 25 has the ADI amplification of Eq. 1."""
    P, u = problem()
    a = b = u
    for n in range(4):
        a = S.orig_dy_step(P, a)
        b = S.orig_adi_step(P, b, n)
    assert energy_norm_rel(a, b) <= 1e-12


def test_fundamental_dyakonov_reproduces_dyakonov():
    """Eqs. 26-27 (the FADI iteration with the procedure) give Eq. 25's fields, and
    u* = 2 v^{n+1/2} (Eq. 28)."""
    P, u0 = problem(5)
    vm = S.fast_dy_init(P, u0)
    u = u0
    ref = u0
    for _ in range(4):
        tau = P.dt / 2
        w = S.add(ref, S.apply_op(P.grid, P.mat, "B", ref), tau)
        ustar = S.solve_implicit(P.grid, P.mat, "A", tau, S.add(w, S.apply_op(P.grid, P.mat, "A", w), tau))
        ref = S.solve_implicit(P.grid, P.mat, "B", tau, ustar)
        u, vm = S.fast_dy_step(P, u, vm)
        assert energy_norm_rel(S.scale(vm, 2.0), ustar) <= 1e-12
        assert energy_norm_rel(u, ref) <= 1e-12


def test_douglas_gunn_steps_like_adi_and_maps_to_fadi():
    """Eq. 29 has the ADI amplification, and its increments are the FADI solves of
    Eq. 30: du* = u~^{n+1/2} - u~^n, du = (u~^{n+1} - u~^n)/2 with u~ = 2u (Eq. 7)."""
    P, u0 = problem(7)
    v = S.fadi_init(P, u0)
    u = u0
    for n in range(3):
        u_dg, dus, du = S.orig_dg_step(P, u)
        assert energy_norm_rel(u_dg, S.orig_adi_step(P, u, n)) <= 1e-12
        vh, wA, _ = S.procedure(P, v, "A", P.dt)
        v1, wB, hB = S.procedure(P, vh, "B", P.dt)
        ut_n = S.scale(u, 2.0)
        # E components: u~^{n+1/2} and u~^{n+1} are the solves w_A, w_B
        for c in G.E_COMPS:
            np.testing.assert_allclose(dus[c], wA[c] - ut_n[c], rtol=0, atol=1e-12 * np.abs(ut_n[c]).max())
            np.testing.assert_allclose(du[c], 0.5 * (wB[c] - ut_n[c]), rtol=0, atol=1e-12 * np.abs(ut_n[c]).max())
        v = v1
        u = u_dg
