"""Quantities the mathematics fixes, used to pin the oracle.

* Field energy  W(u) = 1/2 dV sum(eps E^2 + mu H^2).  A and B (Eqs. 33-34)
  are skew-adjoint in the inner product <u, w> = dV sum(eps E.E' + mu H.H')
  (with PEC walls summation by parts is exact), so every procedure of a
  fundamental scheme, (I + h/2 O)(I - h/2 O)^{-1}, is a Cayley transform and
  conserves W of what it acts on: FLOD/FSS conserve W(u); FADI conserves
  W(v) of its auxiliary state (v^n = (I + dt/2 B) u^n, from Eqs. 2a and 8a).
  The paper asserts unconditional stability (title, Sec. I); this is the
  exact form of it the tests check.
* The discrete dispersion relation of ADI (and LOD1, whose amplification is
  similar to ADI's): with P = (c dt/dx)^2 sin^2(kx dx/2) and Q, R likewise,
      sin^2(w dt / 2) = (P+Q+R+PQ+QR+RP) / ((1+P)(1+Q)(1+R)).
  Derived here from the 6x6 Fourier symbol (checked numerically by a test
  that builds that symbol independently).
"""
from __future__ import annotations

import math

import numpy as np

from .grid import C0, E_COMPS, H_COMPS, Grid


def energy(grid: Grid, mat: dict, u: dict) -> float:
    dv = grid.cell_volume()
    s = 0.0
    for c in E_COMPS + H_COMPS:
        s += float(np.sum(mat[c] * u[c] * u[c]))
    return 0.5 * dv * s


def adi_omega(dt: float, kx: float, ky: float, kz: float, dx: float, dy: float, dz: float,
              c: float = C0, order: int = 2) -> float:
    """Angular frequency of the ADI/LOD1 amplification for wave vector k.
    P = (c dt kappa_x / 2)^2 with kappa the symbol of the staggered first
    difference: (2/d) sin(k d/2) (Yee), or (2/d)(9/8 sin(k d/2) - 1/24 sin(3 k d/2))
    for the fourth-order difference."""
    def kap(k, d):
        if order == 4:
            return (2.0 / d) * (9.0 / 8.0 * math.sin(k * d / 2) - 1.0 / 24.0 * math.sin(1.5 * k * d))
        return (2.0 / d) * math.sin(k * d / 2)
    P = (c * dt * kap(kx, dx) / 2) ** 2
    Q = (c * dt * kap(ky, dy) / 2) ** 2
    R = (c * dt * kap(kz, dz) / 2) ** 2
    s2 = (P + Q + R + P * Q + Q * R + R * P) / ((1 + P) * (1 + Q) * (1 + R))
    return 2.0 * math.asin(math.sqrt(s2)) / dt


def yee_omega(kx, ky, kz, dx, dy, dz, c: float = C0) -> float:
    """Semi-discrete (exact-in-time) angular frequency c |k'| of the Yee grid."""
    kp2 = sum((2.0 / d * math.sin(k * d / 2)) ** 2 for k, d in ((kx, dx), (ky, dy), (kz, dz)))
    return c * math.sqrt(kp2)


def fourier_symbols(kx, ky, kz, dx, dy, dz, eps, mu):
    """6x6 symbols of A and B for a plane wave exp(i k.r) on the Yee grid: every
    staggered first difference d_xi becomes i*kappa_xi, kappa = (2/d) sin(k d/2).
    Component order (Ex, Ey, Ez, Hx, Hy, Hz); rows/columns follow Eqs. 33-34."""
    ix = 1j * (2.0 / dx) * math.sin(kx * dx / 2)
    iy = 1j * (2.0 / dy) * math.sin(ky * dy / 2)
    iz = 1j * (2.0 / dz) * math.sin(kz * dz / 2)
    A = np.zeros((6, 6), dtype=complex)
    B = np.zeros((6, 6), dtype=complex)
    EX, EY, EZ, HX, HY, HZ = range(6)
    A[EX, HZ] = iy / eps; A[EY, HX] = iz / eps; A[EZ, HY] = ix / eps
    A[HX, EY] = iz / mu; A[HY, EZ] = ix / mu; A[HZ, EX] = iy / mu
    B[EX, HY] = -iz / eps; B[EY, HZ] = -ix / eps; B[EZ, HX] = -iy / eps
    B[HX, EZ] = -iy / mu; B[HY, EX] = -iz / mu; B[HZ, EY] = -ix / mu
    return A, B


def adi_amplification(dt, A, B):
    """(I - dt/2 B)^{-1} (I + dt/2 A) (I - dt/2 A)^{-1} (I + dt/2 B)  (Eq. 1)."""
    I = np.eye(A.shape[0])
    t = dt / 2
    return (np.linalg.solve(I - t * B, I + t * A) @ np.linalg.solve(I - t * A, I + t * B))


def lod1_amplification(dt, A, B):
    """(I - dt/2 B)^{-1} (I + dt/2 B) (I - dt/2 A)^{-1} (I + dt/2 A)  (Eq. 11)."""
    I = np.eye(A.shape[0])
    t = dt / 2
    return (np.linalg.solve(I - t * B, I + t * B) @ np.linalg.solve(I - t * A, I + t * A))


def project(u: dict, shape: dict) -> float:
    """<E, shape> summed over the three E components (unit weights)."""
    return float(sum(np.sum(u[c] * shape[c]) for c in E_COMPS))


def fit_cos_omega_dt(a: np.ndarray) -> float:
    """Least-squares fit of a[n+1] + a[n-1] = 2 cos(w dt) a[n] + kappa over a
    time series; returns cos(w dt).  kappa absorbs a static component."""
    a = np.asarray(a, dtype=np.float64)
    y = a[2:] + a[:-2]
    X = np.stack([2.0 * a[1:-1], np.ones_like(a[1:-1])], axis=1)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    return float(coef[0])
