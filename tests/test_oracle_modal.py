"""Pins for the closed-form cavity-mode evolution (oracle/modal.py): it must
reproduce the structured oracle's stepper on small cavities, so that it can
stand in for the oracle at full size."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import modal as M
from oracle import schemes as S

from test_oracle_schemes import rel


@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss"])
def test_modal_closed_form_equals_stepper(scheme):
    nx, ny, nz = 10, 8, 6
    d = (1e-3, 1.2e-3, 0.9e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 6.0 * g.dt_cfl()
    modes = W.random_modes(3, nx, ny, nz, *d, count=3, mmax=5)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    steps = 25
    ref, _, _ = S.run_fundamental(S.Problem(g, dt), scheme, u0, steps)
    got = M.field_after(g, dt, scheme, modes, steps)
    assert rel(got, ref) < 1e-12


def test_modal_initial_field_is_the_workload_field():
    nx, ny, nz = 9, 7, 5
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    modes = W.random_modes(4, nx, ny, nz, 1e-3, 1e-3, 1e-3, count=4, mmax=4)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    got = M.field_after(g, 1e-12, "fadi", modes, 0)
    for c in ("ex", "ey", "ez"):
        assert np.max(np.abs(got[c] - u0[c])) < 1e-14
    for c in ("hx", "hy", "hz"):
        assert np.max(np.abs(got[c])) == 0.0


def test_mode_operators_sum_to_curl_eigenproblem():
    """(A + B) on a mode has eigenvalues 0, 0 and +-i c |kappa| (twice): the
    semi-discrete Yee frequencies."""
    from oracle import invariants as I
    g = G.Grid(12, 10, 8, 1e-3, 1.1e-3, 0.9e-3)
    A, B = M.mode_operators(g, 3, 2, 5)
    ev = np.sort(np.abs(np.linalg.eigvals(A + B).imag))
    w = I.yee_omega(3 * np.pi / (12e-3), 2 * np.pi / (11e-3), 5 * np.pi / (7.2e-3), 1e-3, 1.1e-3, 0.9e-3)
    assert ev[0] < 1e-3 * w and ev[1] < 1e-3 * w
    assert np.allclose(ev[2:], w, rtol=1e-12)
