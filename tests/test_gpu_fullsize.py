"""Full-size parity: cavity-mode workloads at their real sizes and step counts
against the exact closed-form modal evolution of the oracle (oracle/modal.py,
pinned to the stepper in test_oracle_modal.py), element by element; the
eps-block dipole recipe (FLOD, FSS) and every instance of the 64-cavity batch
at their full sizes against the FP64 oracle stepper over the steps it
finishes in about a minute.

Also checks the exactly conserved FADI invariant W(v) at full size."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import modal as M

from gpu_helpers import energy_norm_rel, per_comp_rel

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-4}


def report(name, **kw):
    print(f"\nFULLSIZE {name} " + json.dumps(kw))


def run_cavity(n, steps, prec, cfl=4.0, seed=2, scheme="fadi"):
    from paper_2011_14043_gb300 import Simulation
    d = 1e-3
    g = G.Grid(n, n, n, d, d, d)
    dt = cfl * g.dt_cfl()
    modes = W.random_modes(seed, n, n, n, d, d, d, count=8)
    u0 = W.mode_sum_fields(modes, n, n, n)
    sim = Simulation(n, n, n, d, scheme=scheme, precision=prec, dt=dt)
    sim.set_fields(u0)
    e_init = sim.energy()            # (physical, state invariant) after initialization
    sim.step(steps)
    e_end = sim.energy()
    out = {c: sim.get_field(c) for c in G.COMPS}
    sim.close()
    ref = M.field_after(g, dt, scheme, modes, steps)
    return out, ref, e_init, e_end


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_cavity_128_fadi_1000_steps(prec):
    """128^3 PEC cavity, 1 mm, CFL 4, 8 seeded modes, 1000 FADI steps."""
    out, ref, e0, e1 = run_cavity(128, 1000, prec)
    err = energy_norm_rel(out, ref)
    drift = abs(e1[1] / e0[1] - 1.0)
    report(f"cavity128_fadi_{prec}", rel_err=err, invariant_drift=drift,
           per_comp=per_comp_rel(out, ref))
    assert err <= TOL[prec]
    assert drift <= (1e-12 if prec == "f64" else 1e-4)


def test_cavity_256_fadi_1000_steps_f32():
    """The benchmark workload: 256^3, 1000 FADI steps in FP32 vs the exact field."""
    out, ref, e0, e1 = run_cavity(256, 1000, "f32")
    err = energy_norm_rel(out, ref)
    drift = abs(e1[1] / e0[1] - 1.0)
    report("cavity256_fadi_f32", rel_err=err, invariant_drift=drift, per_comp=per_comp_rel(out, ref))
    assert err <= TOL["f32"]
    assert drift <= 1e-4


@pytest.mark.parametrize("scheme", ["flod", "fss"])
def test_cavity_128_flod_fss_f32(scheme):
    out, ref, e0, e1 = run_cavity(128, 300, "f32", cfl=8.0, scheme=scheme)
    err = energy_norm_rel(out, ref)
    drift = abs(e1[0] / e0[0] - 1.0)
    report(f"cavity128_{scheme}_f32", rel_err=err, energy_drift=drift)
    assert err <= TOL["f32"]
    assert drift <= 1e-4


def run_blocks(n, steps, prec, scheme, seed=3):
    """256^3-type dipole run: eps_r blocks in [1, 10], 0.5 mm cells, CFL 8, z dipole at the centre."""
    from paper_2011_14043_gb300 import Simulation
    d = 0.5e-3
    g = G.Grid(n, n, n, d, d, d)
    dt = 8.0 * g.dt_cfl()
    eps = W.eps_blocks(seed, n, n, n, 1.0, 10.0)
    cur = W.dipole_current((np.arange(steps) + 0.5) * dt)
    sim = Simulation(n, n, n, d, scheme=scheme, precision=prec, dt=dt)
    sim.set_material(eps)
    sim.set_source("ez", n // 2, n // 2, n // 2, cur)
    sim.step(steps)
    out = {c: sim.get_field(c).astype(np.float64) for c in G.COMPS}
    sim.close()
    return out


@pytest.mark.parametrize("scheme", ["flod", "fss"])
def test_blocks_256_f32_vs_f64(scheme):
    """FP32 precision statement at the full 256^3 eps-block dipole size: FP32 fields vs the
    FP64 path (itself pinned to the oracle to 1e-12 on the same recipe at
    reduced size in test_gpu_parity.py)."""
    f64 = run_blocks(256, 1000, "f64", scheme)
    f32 = run_blocks(256, 1000, "f32", scheme)
    err = energy_norm_rel(f32, f64)
    report(f"blocks256_{scheme}_f32_vs_f64", rel_err=err)
    assert err <= 1e-4


def run_batch(wls, prec, steps):
    from paper_2011_14043_gb300 import Batch, Simulation
    sims = []
    for w in wls:
        s = Simulation(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, scheme="fadi", precision=prec, cfl=w.cfl)
        s.set_material(w.eps_r)
        s.set_fields(w.fields)
        sims.append(s)
    b = Batch(sims)
    b.step(steps)
    out = [{c: s.get_field(c).astype(np.float64) for c in G.COMPS} for s in sims]
    dts = [s.dt for s in sims]
    b.close()
    for s in sims:
        s.close()
    return out, dts


def test_batch_64_cavities_500_steps():
    """The 64-cavity batch at full size: 64 seeded cavities of uneven sizes, CFL numbers
    and eps_r blocks, 500 FADI steps as one batch.  Every FP32 instance within
    1e-4 of the FP64 batch; the FP64 batch against the FP64 oracle (structured
    stepper) on the smallest instance over all 500 steps, to 1e-12."""
    from oracle import schemes as S
    wls = W.workload_batch(seed=4, count=64, steps=500)
    f64, dts = run_batch(wls, "f64", 500)
    f32, _ = run_batch(wls, "f32", 500)
    errs = [energy_norm_rel(a, b) for a, b in zip(f32, f64)]
    small = min(range(len(wls)), key=lambda i: wls[i].nx * wls[i].ny * wls[i].nz)
    w = wls[small]
    g = G.Grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    P = S.Problem(g, dts[small], eps_r_cell=w.eps_r)
    ref, _, _ = S.run_fundamental(P, "fadi", w.fields, 500)
    err_oracle = energy_norm_rel(f64[small], ref)
    report("batch64_fadi", max_rel_err_f32_vs_f64=max(errs), median=float(np.median(errs)),
           smallest=[w.nx, w.ny, w.nz], f64_vs_oracle=err_oracle)
    assert max(errs) <= 1e-4
    assert err_oracle <= 1e-12


def oracle_blocks(n, steps, scheme, seed=3):
    """The FP64 oracle on the eps-block dipole recipe (zero initial field)."""
    from oracle import schemes as S
    from gpu_helpers import oracle_problem
    d = 0.5e-3
    g = G.Grid(n, n, n, d, d, d)
    dt = 8.0 * g.dt_cfl()
    eps = W.eps_blocks(seed, n, n, n, 1.0, 10.0)
    cur = W.dipole_current((np.arange(steps) + 0.5) * dt)
    P = oracle_problem(n, n, n, d, d, d, dt, eps=eps, source=("ez", n // 2, n // 2, n // 2, cur))
    ref, _, _ = S.run_fundamental(P, scheme, W.zero_fields(n, n, n), steps)
    return ref


def check_components(out, ref, tol, floor=1e-4):
    """Every component carrying at least `floor` of the energy within `tol`
    relative L2 of the oracle's, and the whole field in the energy norm."""
    err = energy_norm_rel(out, ref)
    comps = per_comp_rel(out, ref, floor=floor)
    assert err <= tol, err
    for c, e in comps.items():
        assert e <= tol, (c, e)
    return err, comps


@pytest.mark.parametrize("scheme", ["flod", "fss"])
def test_blocks_256_vs_oracle(scheme):
    """The full FLOD / FSS recipe (256^3, 0.5 mm cells, eps_r blocks U[1,10],
    CFL 8, z dipole at the centre; Eqs. 15 and 17) element by element against
    the FP64 oracle after 10 steps (what the numpy oracle finishes in about a
    minute on the host): FP64 to 1e-12 and FP32 to 1e-4, the whole field and
    every component carrying at least 1e-4 of the energy."""
    steps = 10
    ref = oracle_blocks(256, steps, scheme)
    res = {}
    for prec in ("f64", "f32"):
        out = run_blocks(256, steps, prec, scheme)
        res[prec] = check_components(out, ref, TOL[prec])
    report(f"blocks256_{scheme}_vs_oracle", steps=steps,
           f64=res["f64"][0], f32=res["f32"][0], f32_per_comp=res["f32"][1])


def test_batch_64_every_instance_vs_oracle():
    """Every one of the 64 cavities of the batch (uneven sizes, CFL numbers and
    eps_r blocks, 8-mode field) against the FP64 oracle after 5 FADI steps of
    the batch: FP64 to 1e-12 and FP32 to 1e-4 per instance, whole field and
    every component carrying at least 1e-4 of the energy."""
    from oracle import schemes as S
    steps = 5
    wls = W.workload_batch(seed=4, count=64, steps=500)
    f64, dts = run_batch(wls, "f64", steps)
    f32, _ = run_batch(wls, "f32", steps)
    worst = {"f64": 0.0, "f32": 0.0}
    for q, w in enumerate(wls):
        g = G.Grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
        P = S.Problem(g, dts[q], eps_r_cell=w.eps_r)
        ref, _, _ = S.run_fundamental(P, "fadi", w.fields, steps)
        for prec, out in (("f64", f64[q]), ("f32", f32[q])):
            err, _ = check_components(out, ref, TOL[prec])
            worst[prec] = max(worst[prec], err)
    report("batch64_every_instance_vs_oracle", steps=steps, worst_f64=worst["f64"], worst_f32=worst["f32"])
