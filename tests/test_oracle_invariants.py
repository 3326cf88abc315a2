"""Pins for the oracle from properties the mathematics fixes.

* Unconditional stability in its exact form: every procedure is a Cayley
  transform of an operator that is skew in the energy product, so FLOD/FSS
  conserve W(u) and FADI conserves W(v) to roundoff at any CFL number.
* Discrete dispersion: the ADI/LOD1 closed form against the eigenvalues of
  the 6x6 Fourier symbol, and PEC-cavity mode frequencies measured from
  oracle runs against the closed form.
* Temporal order: ADI second order in dt; LOD1 fields first order (Table I).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import invariants as I
from oracle import schemes as S

from test_oracle_schemes import make_problem, rel


@pytest.mark.parametrize("cfl", [4.0, 8.0, 10.0])
@pytest.mark.parametrize("scheme", ["flod", "fss", "fadi"])
def test_energy_conserved_at_large_cfl(scheme, cfl):
    P, u0 = make_problem(50, nx=7, ny=6, nz=5, cfl=cfl)
    g = P.grid
    if scheme == "fadi":
        v = S.fadi_init(P, u0)
        e0 = I.energy(g, P.mat, v)
        for n in range(40):
            v = S.fadi_step(P, v, n)
        e1 = I.energy(g, P.mat, v)
    else:
        step = S.flod_step if scheme == "flod" else S.fss_step
        e0 = I.energy(g, P.mat, u0)
        u = u0
        for n in range(40):
            u = step(P, u, n)
        e1 = I.energy(g, P.mat, u)
    assert abs(e1 / e0 - 1) < 1e-12


def test_energy_grows_if_a_coupling_sign_is_flipped():
    """Guard for the guard: the energy test must be able to fail.  Flipping the
    sign of one explicit H update breaks skew-symmetry and the energy drifts."""
    P, u0 = make_problem(51, nx=6, ny=6, nz=6, cfl=4.0)
    g = P.grid
    ec, hc, ax, sg = G.PAIRS["A"][0]
    e0 = I.energy(g, P.mat, u0)
    u = u0
    for n in range(20):
        new, w, hb = S.procedure(P, u, "A", P.dt)
        d = P.dt / (2 * P.mat[hc])
        new[hc] = hb[hc] - sg * d * G.diff_e_to_h(w[ec], G.AXIS[ax], g.spacing[ax])
        u, _, _ = S.procedure(P, new, "B", P.dt)
    assert abs(I.energy(g, P.mat, u) / e0 - 1) > 1e-6


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_dispersion_closed_form_matches_fourier_symbol(seed):
    rng = np.random.default_rng(seed)
    dx, dy, dz = 1e-3, 1.4e-3, 0.7e-3
    k = rng.uniform(0, math.pi, 3) / np.array([dx, dy, dz])
    for cfl in (0.5, 4.0, 10.0):
        dt = cfl / (G.C0 * math.sqrt(dx ** -2 + dy ** -2 + dz ** -2))
        A, B = I.fourier_symbols(*k, dx, dy, dz, G.EPS0, G.MU0)
        for amp in (I.adi_amplification(dt, A, B), I.lod1_amplification(dt, A, B)):
            ev = np.linalg.eigvals(amp)
            assert np.allclose(np.abs(ev), 1.0, atol=1e-12)
            ph = np.sort(np.abs(np.angle(ev)))
            w = I.adi_omega(dt, *k, dx, dy, dz)
            # two static eigenvalues 1, then the doubly degenerate pair exp(+-i w dt)
            assert ph[0] < 1e-7 and ph[1] < 1e-7
            assert np.allclose(ph[2:], w * dt, rtol=1e-10, atol=0)


@pytest.mark.parametrize("scheme", ["fadi", "flod"])
def test_cavity_mode_frequency_matches_closed_form(scheme):
    nx, ny, nz = 10, 8, 6
    dx, dy, dz = 1e-3, 1.2e-3, 0.9e-3
    g = G.Grid(nx, ny, nz, dx, dy, dz)
    P = S.Problem(g, 4.0 * g.dt_cfl())
    modes = W.random_modes(5, nx, ny, nz, dx, dy, dz, count=2, mmax=5)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    u0 = {c: u0[c] for c in G.COMPS}
    shapes = [W.mode_e_shape(m, nx, ny, nz, unit_amp=True) for m in modes]
    steps = 50
    series = np.zeros((len(modes), steps + 1))
    for q, sh in enumerate(shapes):
        series[q, 0] = I.project(u0, sh)
    if scheme == "fadi":
        v = S.fadi_init(P, u0)
        for n in range(steps):
            v, u = S.fadi_step(P, v, n, want_output=True)
            for q, sh in enumerate(shapes):
                series[q, n + 1] = I.project(u, sh)
    else:
        u = u0
        for n in range(steps):
            u = S.flod_step(P, u, n)
            for q, sh in enumerate(shapes):
                series[q, n + 1] = I.project(u, sh)
    for q, m in enumerate(modes):
        kx, ky, kz = m.m * math.pi / (nx * dx), m.n * math.pi / (ny * dy), m.p * math.pi / (nz * dz)
        c_fit = I.fit_cos_omega_dt(series[q])
        w_ref = I.adi_omega(P.dt, kx, ky, kz, dx, dy, dz)
        assert c_fit == pytest.approx(math.cos(w_ref * P.dt), abs=1e-9)


def test_adi_frequency_error_is_second_order():
    """ADI frequency vs the semi-discrete Yee frequency: error ~ dt^2."""
    dx = dy = dz = 1e-3
    k = (3 * math.pi / 0.016, 2 * math.pi / 0.016, math.pi / 0.016)
    ws = I.yee_omega(*k, dx, dy, dz)
    dts = [4e-13, 2e-13, 1e-13]
    errs = [abs(I.adi_omega(dt, *k, dx, dy, dz) - ws) for dt in dts]
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.02)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.02)


def test_lod1_fields_first_order_adi_second_order():
    """At a fixed final time, ||FLOD - FADI|| halves with dt (first order,
    Table I), while FADI's self-convergence error quarters (second order)."""
    nx, ny, nz = 8, 7, 6
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    modes = W.random_modes(9, nx, ny, nz, 1e-3, 1e-3, 1e-3, count=3, mmax=3)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    T = 16 * 0.5 * g.dt_cfl()
    res = {}
    for steps in (32, 64, 128, 256):
        P = S.Problem(g, T / steps)
        ua, _, _ = S.run_fundamental(P, "fadi", u0, steps)
        ul, _, _ = S.run_fundamental(P, "flod", u0, steps)
        res[steps] = (ua, ul)
    d1 = [rel(res[s][1], res[s][0]) for s in (64, 128, 256)]
    assert d1[0] / d1[1] == pytest.approx(2.0, rel=0.08)
    assert d1[1] / d1[2] == pytest.approx(2.0, rel=0.08)
    e = [rel(res[s][0], res[256][0]) for s in (32, 64)]
    # e(dt) ~ C (dt^2 - dt_256^2): (64 - 1)/(16 - 1) = 4.2
    assert e[0] / e[1] == pytest.approx(4.2, rel=0.08)
