"""Pins for the oracle's Thomas solver: dense LU and the closed-form spectrum."""
import math

import numpy as np
import pytest

from oracle.tridiag import thomas, tridiag_dense


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_thomas_matches_dense_lu(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(5):
        # row-scaled symmetric systems like the FDTD lines: diag 1/(2b_j) + (d_-+d_+)/2
        b = rng.uniform(0.05, 2.0, n)
        dfa = rng.uniform(0.1, 3.0, n + 1)
        lower = -b * dfa[:-1] / 2
        upper = -b * dfa[1:] / 2
        diag = 0.5 + b * (dfa[:-1] + dfa[1:]) / 2
        rhs = rng.standard_normal(n)
        x = thomas(lower, diag, upper, rhs)
        m = tridiag_dense(lower, diag, upper)
        ref = np.linalg.solve(m, rhs)
        assert np.max(np.abs(x - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_thomas_batched_axes_independent():
    rng = np.random.default_rng(7)
    shape = (3, 4, 9)
    lower = rng.uniform(-1, 0, shape)
    upper = rng.uniform(-1, 0, shape)
    diag = 2.5 + rng.uniform(0, 1, shape)
    rhs = rng.standard_normal(shape)
    x = thomas(lower, diag, upper, rhs)
    for a in range(3):
        for b in range(4):
            ref = np.linalg.solve(tridiag_dense(lower[a, b], diag[a, b], upper[a, b]), rhs[a, b])
            assert np.allclose(x[a, b], ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,alpha", [(7, 0.3), (31, 2.0), (63, 10.0)])
def test_thomas_constant_coefficients_sine_transform(n, alpha):
    """For the constant-coefficient line system of a homogeneous medium,
    1/2 w_j - alpha (w_{j+1} - 2 w_j + w_{j-1}) = r_j with w_0 = w_{n+1} = 0,
    the discrete sine vectors s_m(j) = sin(m pi j/(n+1)) are eigenvectors with
    eigenvalue 1/2 + 4 alpha sin^2(m pi / (2(n+1))).  Solve r = s_m and compare."""
    j = np.arange(1, n + 1)
    for m in (1, n // 2 + 1, n):
        s = np.sin(m * math.pi * j / (n + 1))
        lam = 0.5 + 4 * alpha * math.sin(m * math.pi / (2 * (n + 1))) ** 2
        x = thomas(np.full(n, -alpha), np.full(n, 0.5 + 2 * alpha), np.full(n, -alpha), s)
        assert np.max(np.abs(x - s / lam)) < 1e-13


def test_thomas_empty_system():
    x = thomas(np.zeros((2, 0)), np.zeros((2, 0)), np.zeros((2, 0)), np.zeros((2, 0)))
    assert x.shape == (2, 0)
