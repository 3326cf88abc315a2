"""Pins for the oracle's source term (the paper omits sources, Sec. II).

The schemes' reading of a point current (weights per procedure, sampling
times) is pinned against something other than itself: the semi-discrete Yee
system dE/dt = (1/eps) curl H - J/eps, dH/dt = -(1/mu) curl E integrated by
RK4 at a small step (``oracle.semidiscrete``).

* The reference itself: RK4 is fourth order; it matches the closed-form
  evolution of a cavity mode (exp of the mode's 6 x 6 operator); and with a
  current it obeys the discrete Poynting theorem dW/dt = -I E_s l_s, which
  fixes the forcing's sign and scale independently of the schemes.
* Every scheme converges to it as dt -> 0 at a fixed final time, at the
  temporal order of Table I: LOD1/FLOD first, ADI/FADI, SS2/FSS and
  LOD2/FLOD2 second.
* Planted mistakes in the oracle's source term fail those checks: a doubled
  weight stops convergence altogether, and sampling the current at t_n
  instead of t_n + dt/2 drops the second-order schemes to first order.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import grid as G
from oracle import invariants as I
from oracle import modal as M
from oracle import schemes as S
from oracle import semidiscrete as SD

NX, NY, NZ = 6, 5, 7
F0, SIG, T0 = 15e9, 25e-12, 60e-12
T_END = 160e-12
STEPS = {"fadi": (40, 80, 160, 320), "flod": (80, 160, 320, 640), "fss": (160, 320, 640),
         "flod2": (40, 80, 160, 320)}
ORDER = {"fadi": 2.0, "flod": 1.0, "fss": 2.0, "flod2": 2.0}


def current(t):
    return math.exp(-((t - T0) / SIG) ** 2) * math.sin(2 * math.pi * F0 * (t - T0))


def setup():
    g = G.Grid(NX, NY, NZ, 1e-3, 1.2e-3, 0.9e-3)
    eps = np.random.default_rng(3).uniform(1, 4, (NZ, NY, NX))
    src = S.Source("ez", 3, 2, 3, current)
    return g, eps, src


def rel_energy(a, b):
    num = den = 0.0
    for c in G.COMPS:
        w = G.EPS0 if c in G.E_COMPS else G.MU0
        num += w * float(np.sum((a[c] - b[c]) ** 2))
        den += w * float(np.sum(b[c] ** 2))
    return math.sqrt(num / den)


@pytest.fixture(scope="module")
def reference():
    g, eps, src = setup()
    mat = S.Problem(g, 1.0, eps_r_cell=eps).mat
    return SD.rk4(g, mat, src, g.zeros(), T_END, SD.rk4_stable_steps(g, T_END, 0.05))


def errors(scheme, reference):
    g, eps, src = setup()
    out = []
    for n in STEPS[scheme]:
        P = S.Problem(g, T_END / n, eps_r_cell=eps, source=src)
        u, _, _ = S.run_fundamental(P, scheme, g.zeros(), n)
        out.append(rel_energy(u, reference))
    return out


def orders(errs):
    return [math.log2(errs[q] / errs[q + 1]) for q in range(len(errs) - 1)]


# --- the reference ----------------------------------------------------------

def test_rk4_reference_is_fourth_order():
    g, eps, src = setup()
    mat = S.Problem(g, 1.0, eps_r_cell=eps).mat
    runs = [SD.rk4(g, mat, src, g.zeros(), T_END, SD.rk4_stable_steps(g, T_END, c)) for c in (0.4, 0.2, 0.1)]
    e1 = rel_energy(runs[0], runs[2])
    e2 = rel_energy(runs[1], runs[2])
    # e(h) ~ C (h^4 - h_min^4): (256 - 1) / (16 - 1) = 17
    assert e1 / e2 == pytest.approx(17.0, rel=0.1)


def test_rk4_reference_matches_the_cavity_mode_closed_form():
    """Without a current a cavity mode evolves by exp(t (A + B)) of its 6 x 6
    operator (oracle.modal), an exact result of the semi-discrete system."""
    g = G.Grid(8, 7, 6, 1e-3, 1e-3, 1e-3)
    mat = S.Problem(g, 1.0).mat
    m, n, p = 2, 3, 1
    c0 = np.array([0.3, -0.5, 0.7, 1e-3, -2e-3, 5e-4])
    u0 = M.fields_from_modes(g, [(m, n, p, c0)])
    t_end = 40 * g.dt_cfl()
    A, B = M.mode_operators(g, m, n, p)
    exact = M.fields_from_modes(g, [(m, n, p, scipy.linalg.expm(t_end * (A + B)) @ c0)])
    e = [rel_energy(SD.rk4(g, mat, None, u0, t_end, SD.rk4_stable_steps(g, t_end, c)), exact)
         for c in (0.05, 0.025)]
    assert e[1] < 2e-7
    assert e[0] / e[1] == pytest.approx(16.0, rel=0.05)


def test_reference_obeys_the_discrete_poynting_theorem():
    """With a current I on one Ez sample (edge length dz), W(T) - W(0) =
    -int I(t) Ez_s(t) dz dt: the forcing -J/eps with J = I / (dx dy) delivers
    exactly the power of the current against the field."""
    g, eps, src = setup()
    mat = S.Problem(g, 1.0, eps_r_cell=eps).mat
    steps = SD.rk4_stable_steps(g, T_END, 0.05)
    h = T_END / steps
    u = g.zeros()
    es = [0.0]
    for n in range(steps):
        u = SD.rk4(g, mat, src, u, h, 1, t0=n * h)
        es.append(float(u["ez"][src.k, src.j, src.i]))
    t = np.arange(steps + 1) * h
    power = -np.array([current(x) for x in t]) * np.array(es) * g.dz
    if steps % 2:                     # composite Simpson needs an even count
        steps -= 1
        power = power[:-1]
        u = SD.rk4(g, mat, src, g.zeros(), steps * h, steps)
    work = h / 3 * (power[0] + power[-1] + 4 * power[1:-1:2].sum() + 2 * power[2:-1:2].sum())
    w_end = I.energy(g, mat, u)
    assert w_end > 0
    assert w_end == pytest.approx(work, rel=1e-5)


# --- the schemes converge to it at their orders -------------------------------

@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_sourced_run_converges_to_the_semi_discrete_system(scheme, reference):
    errs = errors(scheme, reference)
    p = orders(errs)[-1]
    assert p == pytest.approx(ORDER[scheme], abs=0.15), (errs, orders(errs))
    assert errs[-1] < 0.06


# --- planted mistakes in the oracle's source term must be caught -------------

def _plant(monkeypatch, kind):
    orig = S.Problem.f

    def doubled(self, t):
        f = orig(self, t)
        return None if f is None else S.scale(f, 2.0)

    def at_t_n(self, t):
        return orig(self, t - 0.5 * self.dt)

    monkeypatch.setattr(S.Problem, "f", doubled if kind == "doubled" else at_t_n)


@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_a_doubled_source_weight_is_caught(scheme, reference, monkeypatch):
    _plant(monkeypatch, "doubled")
    errs = errors(scheme, reference)
    p = orders(errs)[-1]
    assert not (abs(p - ORDER[scheme]) <= 0.15 and errs[-1] < 0.06), (errs, orders(errs))
    assert errs[-1] > 0.5


@pytest.mark.parametrize("scheme", ["fadi", "fss", "flod2"])
def test_sampling_the_current_at_t_n_is_caught(scheme, reference, monkeypatch):
    _plant(monkeypatch, "at_t_n")
    errs = errors(scheme, reference)
    p = orders(errs)[-1]
    assert not (abs(p - ORDER[scheme]) <= 0.15 and errs[-1] < 0.06), (errs, orders(errs))
    assert p < ORDER[scheme] - 0.4
