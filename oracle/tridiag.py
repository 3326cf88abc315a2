"""Tridiagonal solver of the oracle: the textbook Thomas algorithm.

The paper (Sec. IV) costs each implicit update as tridiagonal systems solved
with bidiagonal (LU) factors, about 5N flops for order N.  The oracle uses the
plain Thomas elimination written out below, vectorised only across independent
systems (the last axis is the system axis); its arithmetic per system is the
sequential textbook order.
"""
from __future__ import annotations

import numpy as np


def thomas(lower: np.ndarray, diag: np.ndarray, upper: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Solve lower[j] x[j-1] + diag[j] x[j] + upper[j] x[j+1] = rhs[j], j = 0..n-1,
    for every system along the last axis.  lower[..., 0] and upper[..., -1] are
    ignored.  All arguments broadcast to rhs's shape."""
    rhs = np.asarray(rhs, dtype=np.float64)
    n = rhs.shape[-1]
    lower = np.broadcast_to(lower, rhs.shape)
    diag = np.broadcast_to(diag, rhs.shape)
    upper = np.broadcast_to(upper, rhs.shape)
    cp = np.empty(rhs.shape, dtype=np.float64)
    dp = np.empty(rhs.shape, dtype=np.float64)
    if n == 0:
        return dp
    # forward elimination
    cp[..., 0] = upper[..., 0] / diag[..., 0]
    dp[..., 0] = rhs[..., 0] / diag[..., 0]
    for j in range(1, n):
        den = diag[..., j] - lower[..., j] * cp[..., j - 1]
        cp[..., j] = upper[..., j] / den
        dp[..., j] = (rhs[..., j] - lower[..., j] * dp[..., j - 1]) / den
    # back substitution
    x = np.empty(rhs.shape, dtype=np.float64)
    x[..., n - 1] = dp[..., n - 1]
    for j in range(n - 2, -1, -1):
        x[..., j] = dp[..., j] - cp[..., j] * x[..., j + 1]
    return x


def tridiag_dense(lower, diag, upper) -> np.ndarray:
    """Dense matrix of one tridiagonal system (for tests on tiny orders)."""
    n = len(diag)
    m = np.zeros((n, n))
    for j in range(n):
        m[j, j] = diag[j]
        if j > 0:
            m[j, j - 1] = lower[j]
        if j < n - 1:
            m[j, j + 1] = upper[j]
    return m
