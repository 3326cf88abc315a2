"""GPU parity in lossy (conductive) media: the CUDA path through the C ABI
against the FP64 oracle on the same seeded inputs.

The loss -sigma/eps E of dE/dt is split evenly between A and B (the paper's
splitting formulae of Sec. II hold for any linear operators; its A and B of
Sec. III are lossless), so every procedure adds b sigma / 4 to its implicit
diagonal: only the FP64-formed pivots change, on the uniform-table path
(uniform eps and sigma), the per-node path (per-cell sigma) and the general
path (per-cell mu).  Bars: 1e-12 (FP64) and 1e-4 (FP32) relative in the
energy norm over the whole field and per component."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import invariants as I
from oracle import modal as M
from oracle import schemes as S

from gpu_helpers import energy_norm_rel, oracle_problem, per_comp_rel, random_fields

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-4}


def check(a, b, prec, floor=1e-4):
    e = energy_norm_rel(a, b)
    assert e <= TOL[prec], e
    for c, v in per_comp_rel(a, b, floor=floor).items():
        assert v <= TOL[prec], (c, v)
    return e


def run(nx, ny, nz, d, dt, scheme, prec, u0, steps, eps=None, mu=None, sigma=None, source=None, probes=(),
        tune=(0, 0)):
    from paper_2011_14043_gb300 import Simulation
    sim = Simulation(nx, ny, nz, *d, scheme=scheme, precision=prec, dt=dt, tune=tune)
    sim.set_material(eps, mu, sigma)
    sim.set_fields(u0)
    if source is not None:
        sim.set_source(*source)
    pids = [sim.add_probe(*p) for p in probes]
    sim.step(steps)
    out = {c: sim.get_field(c).astype(np.float64) for c in G.COMPS}
    series = [sim.get_probe(p, steps) for p in pids]
    en = sim.energy()
    sim.close()
    return out, series, en


MEDIA = ["uniform", "per_cell", "per_cell_mu"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("media", MEDIA)
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_lossy_vs_oracle(scheme, media, prec):
    """A dipole and a random initial field in a lossy medium, ragged grid,
    every scheme and media path, with a probe (not in FLOD2's case)."""
    nx, ny, nz = 30, 27, 23
    d = (1e-3, 0.9e-3, 1.1e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 5.0 * g.dt_cfl()
    rng = np.random.default_rng(17)
    if media == "uniform":
        eps = np.full((nz, ny, nx), 2.0)
        sigma = np.full((nz, ny, nx), 0.8)
        mu = None
    else:
        eps = W.eps_blocks(17, nx, ny, nz, 1.0, 6.0)
        sigma = rng.uniform(0.0, 1.5, (nz, ny, nx))
        mu = rng.uniform(1.0, 2.5, (nz, ny, nx)) if media == "per_cell_mu" else None
    u0 = random_fields(nx, ny, nz, seed=18)
    steps = 12
    cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 30) * 1e-4
    src = ("ez", 14, 12, 10, cur)
    P0 = oracle_problem(nx, ny, nz, *d, dt, source=src)
    P = S.Problem(g, dt, eps_r_cell=eps, mu_r_cell=mu, source=P0.source, sigma_cell=sigma)
    probes = [("ex", 9, 8, 7)] if scheme != "flod2" else []
    ref, _, series = S.run_fundamental(P, scheme, u0, steps, probes=probes)
    out, got_series, en = run(nx, ny, nz, d, dt, scheme, prec, u0, steps, eps, mu, sigma, src, probes)
    check(out, ref, prec)
    for a, b in zip(got_series, series):
        assert np.max(np.abs(a - b)) <= TOL[prec] * np.max(np.abs(b))
    assert en[0] == pytest.approx(I.energy(g, P.mat, ref), rel=TOL[prec])


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss"])
def test_lossy_graph_steps_bit_identical_to_stream_steps(scheme, prec):
    nx, ny, nz = 26, 21, 19
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 6.0 * g.dt_cfl()
    sigma = np.random.default_rng(3).uniform(0.0, 1.0, (nz, ny, nx))
    u0 = random_fields(nx, ny, nz, seed=4)
    a, _, _ = run(nx, ny, nz, (1e-3,) * 3, dt, scheme, prec, u0, 7, sigma=sigma, tune=(16, 0))
    b, _, _ = run(nx, ny, nz, (1e-3,) * 3, dt, scheme, prec, u0, 7, sigma=sigma, tune=(16, 8))
    for c in G.COMPS:
        assert np.array_equal(a[c], b[c]), c


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lossy_cavity_128_fadi_vs_damped_mode_closed_form(prec):
    """128^3 cavity filled with a homogeneous lossy dielectric (eps_r 2.5,
    sigma 0.05 S/m), 8 seeded modes, CFL 4, 500 FADI steps, against the
    oracle's closed-form modal evolution with the split loss (pinned to the
    stepper); the field energy falls monotonically over the run."""
    from paper_2011_14043_gb300 import Simulation
    n, steps = 128, 500
    d = 1e-3
    g = G.Grid(n, n, n, d, d, d)
    dt = 4.0 * g.dt_cfl()
    eps_r, sigma = 2.5, 0.05
    modes = W.random_modes(2, n, n, n, d, d, d, count=8)
    u0 = W.mode_sum_fields(modes, n, n, n)
    sim = Simulation(n, n, n, d, scheme="fadi", precision=prec, dt=dt)
    sim.set_material(np.full((n, n, n), eps_r), None, np.full((n, n, n), sigma))
    sim.set_fields(u0)
    energies = [sim.energy()[1]]
    for _ in range(5):
        sim.step(steps // 5)
        energies.append(sim.energy()[1])
    out = {c: sim.get_field(c).astype(np.float64) for c in G.COMPS}
    sim.close()
    ref = M.field_after(g, dt, "fadi", modes, steps, eps_r=eps_r, sigma=sigma)
    err = energy_norm_rel(out, ref)
    print(f"\nLOSSY cavity128 {prec} rel_err={err:.3e} energy ratio={energies[-1] / energies[0]:.4f}")
    assert err <= TOL[prec]
    assert all(b < a for a, b in zip(energies, energies[1:]))


def test_lossy_batch_vs_oracle():
    """A batch of lossy cavities (per-cell sigma, eps blocks): every instance
    against the oracle."""
    from paper_2011_14043_gb300 import Batch, Simulation
    rng = np.random.default_rng(9)
    grids = [(20, 17, 15), (24, 13, 18), (16, 22, 12)]
    steps = 6
    for prec in ("f64", "f32"):
        sims, refs = [], []
        for q, (nx, ny, nz) in enumerate(grids):
            g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
            dt = 4.0 * g.dt_cfl()
            eps = W.eps_blocks(q, nx, ny, nz, 1.0, 4.0)
            sigma = rng.uniform(0.0, 1.0, (nz, ny, nx))
            u0 = random_fields(nx, ny, nz, seed=q)
            s = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision=prec, dt=dt)
            s.set_material(eps, None, sigma)
            s.set_fields(u0)
            sims.append(s)
            ref, _, _ = S.run_fundamental(S.Problem(g, dt, eps_r_cell=eps, sigma_cell=sigma), "fadi", u0, steps)
            refs.append(ref)
        b = Batch(sims)
        b.step(steps)
        for s, ref in zip(sims, refs):
            check({c: s.get_field(c).astype(np.float64) for c in G.COMPS}, ref, prec)
        b.close()
        for s in sims:
            s.close()


def test_lossy_limits_are_enforced():
    """FADI and FLOD2 need sigma dt / eps <= 2 (their output relation inverts
    a matrix whose loss diagonal has the opposite sign); FLOD/FSS take any
    sigma; negative sigma is invalid; the reverse pass takes lossless media."""
    from paper_2011_14043_gb300 import FdtdError, Simulation
    n = 12
    g = G.Grid(n, n, n, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    big = np.full((n, n, n), 3.0 * G.EPS0 / dt)       # sigma dt / eps0 = 3
    for scheme, ok in (("fadi", False), ("flod2", False), ("flod", True), ("fss", True)):
        sim = Simulation(n, n, n, 1e-3, scheme=scheme, precision="f64", dt=dt)
        if ok:
            sim.set_material(None, None, big)
            sim.set_fields(random_fields(n, n, n, seed=1))
            sim.step(3)
            e = sim.energy()
            assert e[0] < I.energy(g, G.material_at_samples(g), random_fields(n, n, n, seed=1))
        else:
            with pytest.raises(FdtdError) as err:
                sim.set_material(None, None, big)
            assert err.value.code == -6
        sim.close()
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision="f64", dt=dt)
    with pytest.raises(FdtdError) as err:
        sim.set_material(None, None, -np.ones((n, n, n)))
    assert err.value.code == -1
    sim.close()
    from paper_2011_14043_gb300._lib import lib
    import ctypes
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision="f64", dt=dt, tune=(0, 2))
    sim.set_material(np.full((n, n, n), 2.0), None, np.full((n, n, n), 0.1))
    blk = (ctypes.c_int32 * 6)(2, 4, 2, 4, 2, 4)
    a = ctypes.c_void_p()
    assert lib().fdtd_adj_create(sim._h, blk, 4, 2, ctypes.byref(a)) == -6
    sim.close()
