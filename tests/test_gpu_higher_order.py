"""GPU parity of the fourth-order difference variant (fdtd_set_order(4)):
the CUDA path through the C ABI against the FP64 oracle with fourth-order
staggered differences and PEC images (oracle.grid, order = 4), on the same
seeded inputs.  Bars: 1e-12 (FP64) and 1e-4 (FP32) relative in the energy
norm, whole field and every component carrying at least 1e-4 of the
energy."""
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


def check(a, b, prec):
    e = energy_norm_rel(a, b)
    assert e <= TOL[prec], e
    for c, v in per_comp_rel(a, b, floor=1e-4).items():
        assert v <= TOL[prec], (c, v)
    return e


def run4(dims, d, dt, scheme, prec, u0, steps, eps_r=None, source=None, probes=(), tune=(0, 0)):
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = dims
    sim = Simulation(nx, ny, nz, *d, scheme=scheme, precision=prec, dt=dt, tune=tune)
    sim.set_order(4)
    if eps_r is not None:
        sim.set_material(np.full((nz, ny, nx), eps_r))
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


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_fourth_order_vs_oracle(scheme, prec):
    """Ragged grid, uniform eps_r 2, random initial field and a dipole, a
    probe (FADI's output field w/2 every step), every scheme."""
    nx, ny, nz = 23, 19, 17
    d = (1e-3, 0.9e-3, 1.1e-3)
    g = G.Grid(nx, ny, nz, *d, order=4)
    dt = 6.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=41)
    steps = 9
    cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 30) * 1e-4
    src = ("ez", 11, 9, 8, cur)
    P0 = oracle_problem(nx, ny, nz, *d, dt, source=src)
    P = S.Problem(g, dt, eps_r_cell=np.full((nz, ny, nx), 2.0), source=P0.source)
    probes = [("hy", 7, 8, 5)] if scheme != "flod2" else []
    ref, _, series = S.run_fundamental(P, scheme, u0, steps, probes=probes)
    out, got_series, en = run4((nx, ny, nz), d, dt, scheme, prec, u0, steps, eps_r=2.0, source=src,
                               probes=probes)
    check(out, ref, prec)
    for a, b in zip(got_series, series):
        assert np.max(np.abs(a - b)) <= TOL[prec] * np.max(np.abs(b))
    assert en[0] == pytest.approx(I.energy(g, P.mat, ref), rel=TOL[prec])


@pytest.mark.parametrize("dims", [(2, 2, 1), (3, 2, 2), (5, 4, 1), (9, 3, 4)])
def test_fourth_order_small_and_2d_grids(dims):
    """Lines of 1..8 cells (the images reach across short lines) and the
    2-D TM case (nz = 1)."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3, order=4)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=7)
    ref, _, _ = S.run_fundamental(S.Problem(g, dt), "fadi", u0, 6)
    out, _, _ = run4(dims, (1e-3,) * 3, dt, "fadi", "f64", u0, 6)
    if any(np.any(ref[c]) for c in G.COMPS):
        check(out, ref, "f64")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fourth_order_graph_steps_bit_identical_to_stream_steps(prec):
    nx, ny, nz = 21, 18, 16
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3, order=4)
    dt = 5.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=8)
    a, _, _ = run4((nx, ny, nz), (1e-3,) * 3, dt, "fss", prec, u0, 6, tune=(16, 0))
    b, _, _ = run4((nx, ny, nz), (1e-3,) * 3, dt, "fss", prec, u0, 6, tune=(16, 8))
    for c in G.COMPS:
        assert np.array_equal(a[c], b[c]), c


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme,dims", [("fadi", (23, 19, 17)), ("flod2", (40, 3, 70)),
                                         ("fss", (300, 33, 2)), ("flod", (65, 257, 9)),
                                         ("fadi", (530, 6, 5))])
def test_fourth_order_tiled_kernel_matches_line_kernel(scheme, dims, prec):
    """The block-tiled kernel (lines of up to 512 cells: chunk counts 2, 8
    and 16, ragged tiles, lanes off the walls, converged factor rows in
    registers) against the one-thread-per-line kernel (tune[1] bit 9) on
    the same inputs: the same arithmetic in the same order, so the fields
    agree to the last bit.  Lines longer than 512 cells (530) take the line
    kernel in both runs."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3, order=4)
    dt = 5.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=12)
    a, _, ea = run4(dims, (1e-3,) * 3, dt, scheme, prec, u0, 4, tune=(0, 0))
    b, _, eb = run4(dims, (1e-3,) * 3, dt, scheme, prec, u0, 4, tune=(0, 512))
    for c in G.COMPS:
        assert np.array_equal(a[c], b[c]), (c, float(np.max(np.abs(a[c] - b[c]))))
    assert ea == eb


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fourth_order_cavity_128_vs_modal_closed_form(prec):
    """128^3 PEC cavity, 1 mm, CFL 4, 8 seeded modes, 200 FADI steps with
    fourth-order differences, against the oracle's closed-form modal
    evolution with the fourth-order symbol (pinned to the stepper); the
    invariant is conserved."""
    from paper_2011_14043_gb300 import Simulation
    n, steps = 128, 200
    d = 1e-3
    g = G.Grid(n, n, n, d, d, d, order=4)
    dt = 4.0 * g.dt_cfl()
    modes = W.random_modes(2, n, n, n, d, d, d, count=8)
    u0 = W.mode_sum_fields(modes, n, n, n)
    sim = Simulation(n, n, n, d, scheme="fadi", precision=prec, dt=dt)
    sim.set_order(4)
    sim.set_fields(u0)
    e0 = sim.energy()[1]
    sim.step(steps)
    e1 = sim.energy()[1]
    out = {c: sim.get_field(c).astype(np.float64) for c in G.COMPS}
    sim.close()
    ref = M.field_after(g, dt, "fadi", modes, steps)
    err = energy_norm_rel(out, ref)
    print(f"\nORDER4 cavity128 {prec} rel_err={err:.3e} invariant drift={abs(e1 / e0 - 1):.2e}")
    assert err <= TOL[prec]
    assert abs(e1 / e0 - 1) <= (1e-12 if prec == "f64" else 1e-4)


def test_fourth_order_limits():
    from paper_2011_14043_gb300 import Batch, FdtdError, Simulation
    n = 10
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision="f64", cfl=3.0)
    with pytest.raises(FdtdError) as err:
        sim.set_order(3)
    assert err.value.code == -1
    eps = np.ones((n, n, n))
    eps[2:5, 2:5, 2:5] = 3.0
    sim.set_material(eps)
    with pytest.raises(FdtdError) as err:
        sim.set_order(4)
    assert err.value.code == -6
    sim.close()
    sim = Simulation(n, n, n, 1e-3, scheme="fadi", precision="f64", cfl=3.0)
    sim.set_order(4)
    with pytest.raises(FdtdError) as err:
        sim.set_material(eps)
    assert err.value.code == -6
    with pytest.raises(FdtdError) as err:
        sim.set_material(None, None, np.full((n, n, n), 0.1))
    assert err.value.code == -6
    with pytest.raises(FdtdError) as err:
        Batch([sim])
    assert err.value.code == -6
    sim.step(1)
    with pytest.raises(FdtdError) as err:
        sim.set_order(2)
    assert err.value.code == -7
    sim.close()
