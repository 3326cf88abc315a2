"""Batched stepping of many independent cavities (the 64-cavity recipe at
reduced sizes): every grid against the FP64 oracle and against the same
grid stepped on its own (the batch runs the same arithmetic: bit-identical)."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import schemes as S

from gpu_helpers import energy_norm_rel

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-4}


def small_batch(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    d = 1e-3
    for b in range(count):
        nx = int(rng.integers(6, 40)); ny = int(rng.integers(6, 30)); nz = int(rng.integers(5, 34))
        cfl = float(rng.uniform(2.0, 10.0))
        eps = W.eps_blocks(rng, nx, ny, nz, 1.0, 4.0) if b % 3 else None   # some uniform grids too
        modes = W.random_modes(rng, nx, ny, nz, d, d, d, count=3, mmax=4)
        out.append((nx, ny, nz, cfl, eps, W.mode_sum_fields(modes, nx, ny, nz)))
    return out


def make_sim(spec, scheme, prec):
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz, cfl, eps, u0 = spec
    sim = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision=prec, cfl=cfl)
    if eps is not None:
        sim.set_material(eps)
    sim.set_fields(u0)
    return sim


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss"])
def test_batch_matches_oracle_and_single(scheme, prec):
    from paper_2011_14043_gb300 import Batch
    specs = small_batch(40 + len(scheme), 7)
    steps = 9
    sims = [make_sim(sp, scheme, prec) for sp in specs]
    batch = Batch(sims)
    batch.step(4)
    batch.step(steps - 4)            # a second call replays the same graph
    assert batch.launches_per_step() >= 2
    for sp, sim in zip(specs, sims):
        nx, ny, nz, cfl, eps, u0 = sp
        g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
        ref, _, _ = S.run_fundamental(S.Problem(g, sim.dt, eps_r_cell=eps), scheme, u0, steps)
        got = sim.get_fields()
        assert energy_norm_rel(got, ref) <= TOL[prec]
        alone = make_sim(sp, scheme, prec)
        alone.step(steps)
        for c in G.COMPS:
            assert np.array_equal(alone.get_field(c), got[c]), c
    batch.close()


def test_batch_rejects_mixed_and_sourced():
    from paper_2011_14043_gb300 import Batch, FdtdError, Simulation
    a = Simulation(8, 8, 8, 1e-3, scheme="fadi", precision="f32", cfl=2.0)
    b = Simulation(8, 8, 8, 1e-3, scheme="flod", precision="f32", cfl=2.0)
    with pytest.raises(FdtdError):
        Batch([a, b])
    c = Simulation(8, 8, 8, 1e-3, scheme="fadi", precision="f32", cfl=2.0)
    c.set_source("ez", 4, 4, 4, np.ones(3))
    with pytest.raises(FdtdError):
        Batch([a, c])
    with pytest.raises(FdtdError):
        Batch([a, a])
