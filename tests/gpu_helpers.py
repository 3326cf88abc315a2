"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the
FP64 oracle on identical seeded inputs)."""
import math

import numpy as np

from oracle import grid as G
from oracle import schemes as S

COMPS = G.COMPS


def energy_norm_rel(a: dict, b: dict) -> float:
    """Relative error in the energy norm (weights eps0 for E, mu0 for H)."""
    num = den = 0.0
    for c in COMPS:
        w = G.EPS0 if c in G.E_COMPS else G.MU0
        num += w * float(np.sum((np.asarray(a[c], np.float64) - b[c]) ** 2))
        den += w * float(np.sum(b[c] ** 2))
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def per_comp_rel(a: dict, b: dict, floor: float = 1e-6) -> dict:
    """Relative L2 per component, for components carrying > floor of the energy."""
    tot = {c: (G.EPS0 if c in G.E_COMPS else G.MU0) * float(np.sum(b[c] ** 2)) for c in COMPS}
    s = sum(tot.values())
    out = {}
    for c in COMPS:
        if tot[c] > floor * s:
            out[c] = float(np.linalg.norm(np.asarray(a[c], np.float64) - b[c]) / np.linalg.norm(b[c]))
    return out


def gpu_run(nx, ny, nz, dx, dy, dz, dt, scheme, precision, fields, steps, eps=None, source=None,
            probes=(), tune=(0, 0)):
    """Run the CUDA path; returns (fields, probe series, (energy, invariant), sim)."""
    from paper_2011_14043_gb300 import Simulation
    sim = Simulation(nx, ny, nz, dx, dy, dz, scheme=scheme, precision=precision, dt=dt, tune=tune)
    if eps is not None:
        sim.set_material(eps)
    for c in COMPS:
        sim.set_field(c, fields[c])
    if source is not None:
        sim.set_source(*source)
    pids = [sim.add_probe(*p) for p in probes]
    sim.step(steps)
    out = {c: sim.get_field(c).astype(np.float64) for c in COMPS}
    series = [sim.get_probe(p, steps) for p in pids]
    en = sim.energy()
    return out, series, en, sim


def oracle_problem(nx, ny, nz, dx, dy, dz, dt, eps=None, source=None):
    src = None
    if source is not None:
        comp, i, j, k, cur = source
        cur = np.asarray(cur, dtype=np.float64)
        tt = dt

        def current(t, cur=cur, tt=tt):
            n = int(round(t / tt - 0.5))
            return float(cur[n]) if 0 <= n < len(cur) else 0.0
        src = S.Source(comp, k, j, i, current)
    return S.Problem(G.Grid(nx, ny, nz, dx, dy, dz), dt, eps_r_cell=eps, source=src)


def random_fields(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    g = G.Grid(nx, ny, nz, 1, 1, 1)
    u = {}
    for c in COMPS:
        u[c] = rng.standard_normal(g.shape(c))
        if c in G.E_COMPS:
            u[c] *= g.e_interior_mask(c)
        else:
            u[c] /= 376.73
    return u
