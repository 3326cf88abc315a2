"""Pins of the oracle's discrete FADI adjoint (oracle/adjoint.py) against
things other than itself: transpose identities of every linear block, and
central finite differences of the forward objective in FP64."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import grid as G
from oracle import schemes as S
from oracle.tridiag import tridiag_dense

from gpu_helpers import oracle_problem, random_fields


def inner(a: dict, b: dict) -> float:
    return sum(float(np.sum(a[c] * b[c])) for c in a)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_difference_transposes(axis):
    rng = np.random.default_rng(axis)
    e_shape = [5, 6, 7]
    h_shape = list(e_shape)
    h_shape[axis] -= 1
    e = rng.standard_normal(e_shape)
    h = rng.standard_normal(h_shape)
    # diff_e_to_h: E shape -> H shape
    assert np.dot(G.diff_e_to_h(e, axis, 0.7).ravel(), h.ravel()) == pytest.approx(
        np.dot(e.ravel(), AD.diff_e_to_h_T(h, axis, 0.7, e_shape).ravel()), rel=1e-13)
    # diff_h_to_e: H shape -> E shape
    assert np.dot(G.diff_h_to_e(h, axis, 0.7, e_shape).ravel(), e.ravel()) == pytest.approx(
        np.dot(h.ravel(), AD.diff_h_to_e_T(e, axis, 0.7, h_shape).ravel()), rel=1e-13)


def test_transposed_line_solve_against_dense():
    rng = np.random.default_rng(11)
    n = 9
    gE = rng.uniform(0.5, 2.0, (3, n + 1))
    gH = rng.uniform(0.5, 2.0, (3, n))
    lo, ce, up = G.line_operator_coeffs(gE, gH, 1, 0.8)
    r = rng.standard_normal((3, n + 1))
    w = AD.solve_lines_T(0.5, lo, ce, up, r, 1)
    for row in range(3):
        M = tridiag_dense(-lo[row], 0.5 - ce[row], -up[row])
        x = np.linalg.solve(M.T, r[row, 1:-1])
        np.testing.assert_allclose(w[row, 1:-1], x, rtol=1e-12, atol=1e-14)
        assert w[row, 0] == 0.0 and w[row, -1] == 0.0


@pytest.mark.parametrize("op", ["A", "B"])
def test_procedure_adjoint_is_the_transpose(op):
    """<lam, P x> = <P^T lam, x> for one procedure (linear in the state)."""
    nx, ny, nz = 6, 5, 4
    g = G.Grid(nx, ny, nz, 1e-3, 1.1e-3, 0.9e-3)
    eps = np.random.default_rng(3).uniform(1.0, 6.0, (nz, ny, nx))
    P = S.Problem(g, 5.0 * g.dt_cfl(), eps_r_cell=eps)
    x = random_fields(nx, ny, nz, seed=4)
    lam = random_fields(nx, ny, nz, seed=5)
    y, w, _ = S.procedure(P, x, op, P.dt)
    epsbar = {c: np.zeros(g.shape(c)) for c in G.E_COMPS}
    back = AD.procedure_adjoint(P, op, P.dt, x, w, lam, None, None, epsbar)
    assert inner(lam, y) == pytest.approx(inner(back, x), rel=1e-12)


def small_problem(seed=7):
    nx, ny, nz = 6, 5, 5
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 4.0 * g.dt_cfl()
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 6.0, (nz, ny, nx))
    steps = 7
    cur = W.dipole_current((np.arange(steps + 2) + 0.5) * dt * 20) * 1e-3
    src = ("ez", 2, 2, 2, cur)
    u0 = random_fields(nx, ny, nz, seed=seed + 1)
    block = (3, 5, 1, 4, 1, 4)
    return g, dt, eps, src, u0, block, steps


def objective(g, dt, eps, src, u0, block, steps):
    P = oracle_problem(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, dt, eps=eps, source=src)
    return AD.forward(P, u0, steps, AD.probe_masks(g, block))[0]


def test_gradient_matches_central_differences():
    """Every cell's dJ/d eps_r (source, initial field, probe block) against
    central differences of the forward objective."""
    g, dt, eps, src, u0, block, steps = small_problem()
    P = oracle_problem(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, dt, eps=eps, source=src)
    J, grad, _ = AD.gradient(P, u0, steps, AD.probe_masks(g, block))
    assert J == pytest.approx(objective(g, dt, eps, src, u0, block, steps), rel=1e-14)
    fd = np.zeros_like(grad)
    h = 1e-5
    for idx in np.ndindex(eps.shape):
        ep = eps.copy(); ep[idx] += h
        em = eps.copy(); em[idx] -= h
        fd[idx] = (objective(g, dt, ep, src, u0, block, steps) - objective(g, dt, em, src, u0, block, steps)) / (2 * h)
    err = np.linalg.norm(grad - fd) / np.linalg.norm(fd)
    assert err <= 1e-6, err
    # the cells next to the source sample and next to the probe block both matter
    assert np.count_nonzero(np.abs(fd) > 1e-3 * np.abs(fd).max()) > eps.size // 4


def test_cell_gradient_is_the_transpose_of_edge_averaging():
    g = G.Grid(4, 3, 5, 1e-3, 1e-3, 1e-3)
    rng = np.random.default_rng(2)
    er = rng.uniform(1, 3, (5, 3, 4))
    de = rng.standard_normal((5, 3, 4))
    ebar = {c: rng.standard_normal(g.shape(c)) for c in G.E_COMPS}
    m1 = G.material_at_samples(g, er + de)
    m0 = G.material_at_samples(g, er)
    # eps_sample is linear in eps_r: <ebar, M de> = <M^T ebar, de>
    lhs = sum(float(np.sum(ebar[c] * (m1[c] - m0[c]))) for c in G.E_COMPS)
    rhs = float(np.sum(AD.cell_gradient(g, ebar) * de))
    assert lhs == pytest.approx(rhs, rel=1e-12)
