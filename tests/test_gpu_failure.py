"""Failure detection without a GPU fault: a bounded device wait that runs out
(an mbarrier arrival that never comes) gives FDTD_ERR_TIMEOUT through the
device error flag, and the context keeps working afterwards."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TIMEOUT = -4


def test_bounded_wait_runs_out_and_the_context_survives():
    from paper_2011_14043_gb300 import Simulation
    from paper_2011_14043_gb300._lib import lib
    L = lib()
    t0 = time.perf_counter()
    rc = L.fdtd_selftest_bounded_wait(50_000_000, 0, None)     # 50 ms, nobody arrives
    waited = time.perf_counter() - t0
    assert rc == TIMEOUT
    assert 0.045 <= waited < 2.0
    assert L.fdtd_selftest_bounded_wait(50_000_000, 1, None) == 0  # the arrival completes the phase
    # the same context still steps and reads back
    sim = Simulation(16, 12, 10, 1e-3, scheme="fadi", precision="f64", cfl=3.0)
    ez = np.zeros(sim.shape("ez"))
    ez[4:6, 5:7, 7:9] = 1.0
    sim.set_field("ez", ez)
    sim.step(3)
    out = sim.get_field("ez")
    assert np.all(np.isfinite(out)) and np.abs(out).max() > 0
    sim.close()


def run_sequence(prec):
    """A full use of one handle: create, inhomogeneous media, source, probe-free
    stepping (graph path), energy, field read-back (FADI output transform)."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 18, 14, 12
    eps = np.ones((nz, ny, nx))
    eps[3:7, 4:9, 5:12] = 3.0
    sim = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision=prec, cfl=4.0)
    try:
        sim.set_material(eps)
        ez = np.zeros(sim.shape("ez"))
        ez[5, 6, 8] = 1.0
        sim.set_field("ez", ez)
        sim.set_source("ez", 9, 7, 6, np.linspace(0.0, 1e-6, 8))
        sim.step(4)
        e = sim.energy()
        out = sim.get_field("ez")
    finally:
        sim.close()
    return e, out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_injected_allocation_failures_are_reported_and_cleaned_up(prec):
    """Fail each device allocation of the sequence in turn: every failure
    surfaces as FDTD_ERR_OOM (or, for a handle it already poisoned,
    FDTD_ERR_STATE) without a fault, and afterwards the same sequence gives the
    same answer as before."""
    from paper_2011_14043_gb300 import FdtdError
    from paper_2011_14043_gb300._lib import lib
    L = lib()
    ref_e, ref_out = run_sequence(prec)
    outcome = []
    for k in range(80):
        L.fdtd_debug_fail_alloc(k)
        try:
            run_sequence(prec)
            outcome.append(True)
        except FdtdError as err:
            assert err.code in (-2, -7), err
            outcome.append(False)
        finally:
            L.fdtd_debug_fail_alloc(-1)
    # early allocations fail the sequence; past its last allocation it completes
    assert outcome.count(False) >= 8 and all(outcome[-10:])
    e, out = run_sequence(prec)
    assert e == ref_e
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["flod", "fadi"])
def test_invariant_growth_is_reported_as_unstable(scheme, prec):
    """A source-free run conserves the scheme invariant exactly (every
    procedure is a Cayley transform of an energy-skew operator): growth past
    the reference taken when the run started is FDTD_ERR_UNSTABLE.  Growth is
    planted from the host by scaling one E component of the state (a restored
    "checkpoint" that is not one; fdtd_set_state keeps the reference), and a
    legitimate new start (fdtd_set_field) takes a new reference."""
    from paper_2011_14043_gb300 import FdtdError, Simulation
    from gpu_helpers import random_fields
    nx, ny, nz = 20, 18, 16
    u0 = random_fields(nx, ny, nz, seed=5)
    sim = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision=prec, cfl=6.0)
    sim.set_fields(u0)
    sim.step(20)
    e_ok = sim.energy()
    ex = sim.get_state("ex")
    sim.set_state("ex", ex * 1.5)
    sim.step(2)
    with pytest.raises(FdtdError) as err:
        sim.energy()
    assert err.value.code == -5
    # a new start from fields takes a new reference: no error
    sim.set_fields(u0)
    sim.step(20)
    e_again = sim.energy()
    assert e_again[1] == pytest.approx(e_ok[1], rel=1e-12 if prec == "f64" else 1e-4)
    sim.close()
