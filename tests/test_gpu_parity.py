"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Bars: relative error <= 1e-12 in FP64 mode and <= 1e-4
in FP32 mode, in the energy norm over all six components and per component
(every component carrying at least 1e-4 of the energy), for probe series
(relative to the series' maximum) and for energies."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import invariants as I
from oracle import schemes as S

from gpu_helpers import (energy_norm_rel, gpu_run, oracle_problem, per_comp_rel,
                         random_fields)

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-4}


def check(a, b, prec):
    """The whole field in the energy norm and every component carrying at
    least 1e-4 of the energy, each within the stated tolerance."""
    e = energy_norm_rel(a, b)
    assert e <= TOL[prec], e
    for c, v in per_comp_rel(a, b, floor=1e-4).items():
        assert v <= TOL[prec], (c, v)
    return e


def test_2d_gaussian_fadi_f64_vs_original_adi():
    """64 x 64 TM (nz = 1), CFL 5, 200 steps, probe Ez(16,16) vs the original ADI."""
    wl = W.workload_2d_gaussian(seed=1)
    g = G.Grid(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz)
    dt = wl.cfl * g.dt_cfl()
    P = S.Problem(g, dt)
    u = {c: wl.fields[c].copy() for c in G.COMPS}
    probe = np.zeros(wl.steps)
    for n in range(wl.steps):
        u = S.orig_adi_step(P, u, n)
        probe[n] = u["ez"][0, 16, 16]
    out, series, en, _ = gpu_run(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz, dt, "fadi", "f64",
                                 wl.fields, wl.steps, probes=[("ez", 16, 16, 0)])
    check(out, u, "f64")
    assert np.max(np.abs(series[0] - probe)) <= 1e-12 * np.max(np.abs(probe))
    assert en[0] == pytest.approx(I.energy(g, P.mat, u), rel=1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
@pytest.mark.parametrize("dims", [(40, 37, 29), (33, 20, 70)])
def test_3d_schemes_vs_oracle(scheme, prec, dims):
    """Grids spanning several warps/segments with ragged tails on every axis."""
    nx, ny, nz = dims
    d = (1e-3, 0.9e-3, 1.1e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 6.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=sum(dims))
    steps = 12
    P = S.Problem(g, dt)
    ref, _, _ = S.run_fundamental(P, scheme, u0, steps)
    out, _, _, _ = gpu_run(nx, ny, nz, *d, dt, scheme, prec, u0, steps)
    check(out, ref, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["flod", "fss", "fadi"])
def test_inhomogeneous_with_dipole_vs_oracle(scheme, prec):
    """eps_r blocks in [1, 10] and a z-directed dipole (per-node coefficients)."""
    nx, ny, nz = 36, 34, 30
    d = 0.5e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 8.0 * g.dt_cfl()
    eps = W.eps_blocks(3, nx, ny, nz, 1.0, 10.0)
    steps = 30
    cur = W.dipole_current((np.arange(steps) + 0.5) * dt * 20)  # compressed pulse in time
    src = ("ez", nx // 2, ny // 2, nz // 2, cur)
    P = oracle_problem(nx, ny, nz, d, d, d, dt, eps=eps, source=src)
    u0 = W.zero_fields(nx, ny, nz)
    ref, _, _ = S.run_fundamental(P, scheme, u0, steps)
    out, _, en, _ = gpu_run(nx, ny, nz, d, d, d, dt, scheme, prec, u0, steps, eps=eps, source=src)
    check(out, ref, prec)
    assert en[0] == pytest.approx(I.energy(g, P.mat, ref), rel=TOL[prec])


@pytest.mark.parametrize("dims", [(2, 2, 1), (2, 2, 2), (3, 2, 2), (2, 3, 4), (5, 4, 1), (3, 3, 3)])
@pytest.mark.parametrize("scheme", ["fadi", "flod"])
def test_degenerate_tiny_grids(dims, scheme):
    """Lines with zero or one unknown, a single layer, single-warp rows."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 3.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=nx * 100 + ny * 10 + nz)
    P = S.Problem(g, dt)
    ref, _, _ = S.run_fundamental(P, scheme, u0, 5)
    out, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, scheme, "f64", u0, 5)
    check(out, ref, "f64")


@pytest.mark.parametrize("dims", [(300, 3, 3), (3, 300, 3), (3, 3, 300), (1000, 2, 2),
                                  (1024, 3, 3), (3, 1024, 3), (3, 3, 1024)])
def test_long_lines(dims):
    """Long lines along each axis (many segments; x rows up to 32 nodes/lane)."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 10.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=7)
    P = S.Problem(g, dt)
    ref, _, _ = S.run_fundamental(P, "fadi", u0, 4)
    for prec in ("f64", "f32"):
        out, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "fadi", prec, u0, 4)
        check(out, ref, prec)


@pytest.mark.parametrize("L", [8, 16, 32])
def test_segment_length_choices_agree(L):
    """Every y/z segment length gives the oracle's answer (tuning override)."""
    nx, ny, nz = 35, 70, 45
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=L)
    P = S.Problem(g, dt)
    ref, _, _ = S.run_fundamental(P, "fadi", u0, 3)
    out, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "fadi", "f64", u0, 3, tune=(L, 0))
    check(out, ref, "f64")


def test_state_round_trip_and_restart():
    """Checkpoint the raw FADI state, restore it in a new handle, continue: same as straight through."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 20, 18, 16
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=3)
    a = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision="f64", dt=dt)
    a.set_fields(u0)
    a.step(5)
    state = {c: a.get_state(c) for c in G.COMPS}
    a.step(5)
    b = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision="f64", dt=dt)
    for c in G.COMPS:
        b.set_state(c, state[c])
    b.step(5)
    fa = a.get_fields()
    fb = b.get_fields()
    assert energy_norm_rel(fb, fa) == 0.0


def test_set_field_after_steps_reinitialises():
    """Setting a field mid-run re-forms the FADI state from the physical field."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 16, 14, 12
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=5)
    P = S.Problem(g, dt)
    sim = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision="f64", dt=dt)
    sim.set_fields(u0)
    sim.step(3)
    mid = sim.get_fields()
    mid["ez"] = mid["ez"] * 0.5
    sim.set_field("ez", mid["ez"])
    sim.step(3)
    ref, _, _ = S.run_fundamental(P, "fadi", mid, 3)
    check(sim.get_fields(), ref, "f64")


def test_device_buffers_path():
    """set_field/get_field with torch CUDA tensors (on_device = 1)."""
    import torch
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 24, 20, 18
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=9)
    sim = Simulation(nx, ny, nz, 1e-3, scheme="flod", precision="f64", dt=dt)
    for c in G.COMPS:
        sim.set_field(c, torch.from_numpy(u0[c]).cuda())
    sim.step(4)
    out = {c: sim.get_field(c, device=True).cpu().numpy() for c in G.COMPS}
    ref, _, _ = S.run_fundamental(S.Problem(g, dt), "flod", u0, 4)
    check(out, ref, "f64")


@pytest.mark.parametrize("prec", ["f32"])
@pytest.mark.parametrize("dims", [(70, 45, 33), (40, 256, 37), (37, 41, 256)])
def test_tma_path_bit_identical_to_direct_path(prec, dims):
    """The persistent TMA-fed y/z kernel of FP32 fields (register stores by
    default, TMA stores with tune[1] bit 2) and the direct-load kernel run
    the same arithmetic in the same order: results must agree bit for bit."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 7.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=nx + ny + nz)
    a, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "fadi", prec, u0, 3, tune=(16, 0))
    b, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "fadi", prec, u0, 3, tune=(16, 1))
    c2, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "fadi", prec, u0, 3, tune=(16, 4))  # TMA stores
    for c in G.COMPS:
        assert np.array_equal(a[c], b[c]), c
        assert np.array_equal(c2[c], b[c]), c


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_pinned_host_buffers_match_pageable(prec):
    """Fields set from page-locked host memory are read in place by the
    unpacking kernel (no staging copy); pageable memory (and tune[1] bit 8)
    takes the staged copy.  Both give identical arrays, read back into
    pinned or pageable memory alike."""
    import torch
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 37, 29, 23
    dtype = np.float64 if prec == "f64" else np.float32
    tdt = torch.float64 if prec == "f64" else torch.float32
    u0 = random_fields(nx, ny, nz, seed=91)
    outs = []
    for pinned, tune in ((True, (0, 0)), (False, (0, 0)), (True, (0, 256))):
        sim = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision=prec, cfl=4.0, tune=tune)
        for c in G.COMPS:
            if pinned:
                t = torch.empty(u0[c].shape, dtype=tdt, pin_memory=True)
                t.numpy()[...] = u0[c].astype(dtype)
                sim.set_field(c, t.numpy())
            else:
                sim.set_field(c, u0[c].astype(dtype))
        sim.step(5)
        got = {}
        for c in G.COMPS:
            if pinned:
                t = torch.empty(sim.shape(c), dtype=tdt, pin_memory=True)
                sim.get_field(c, out=t.numpy())
                got[c] = t.numpy().copy()
            else:
                got[c] = sim.get_field(c)
        outs.append(got)
        sim.close()
    for c in G.COMPS:
        assert np.array_equal(outs[0][c], outs[1][c]), c
        assert np.array_equal(outs[2][c], outs[1][c]), c


@pytest.mark.parametrize("scheme", ["fadi", "fss"])
@pytest.mark.parametrize("dims", [(256, 40, 33), (200, 37, 29), (129, 20, 24), (256, 9, 300)])
def test_tma_rows_bit_identical_to_direct_rows(dims, scheme):
    """The persistent TMA-fed x-line kernel of FP32 fields in homogeneous
    media (tune[1] bit 4; lines of 129..256 cells; every ring depth and
    blocks-per-SM variant, bits 5-6) against the one-warp-per-line kernel:
    the same arithmetic on the same values, bit for bit; and the oracle's
    answer."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 6.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=nx + 2 * ny + 3 * nz)
    steps = 4
    ref_tma = None
    for bits in (16, 48, 80, 112):
        a, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, scheme, "f32", u0, steps, tune=(0, bits))
        if ref_tma is None:
            ref_tma = a
        for c in G.COMPS:
            assert np.array_equal(a[c], ref_tma[c]), (bits, c)
    b, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, scheme, "f32", u0, steps, tune=(0, 0))
    for c in G.COMPS:
        assert np.array_equal(ref_tma[c], b[c]), c
    ref, _, _ = S.run_fundamental(S.Problem(g, dt), scheme, u0, steps)
    check(ref_tma, ref, "f32")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fadi_probes_at_and_beside_the_source(prec):
    """FADI probe series (the output field w_B/2 of every step) at the source
    sample itself and next to it, against the oracle's output field."""
    nx, ny, nz = 20, 18, 16
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 5.0 * g.dt_cfl()
    eps = W.eps_blocks(9, nx, ny, nz, 1.0, 4.0)
    steps = 40
    cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 15)
    src = ("ez", 10, 9, 8, cur)
    P = oracle_problem(nx, ny, nz, d, d, d, dt, eps=eps, source=src)
    probes = [("ez", 10, 9, 8), ("ez", 11, 9, 8), ("ex", 10, 9, 8)]
    _, _, ref = S.run_fadi(P, W.zero_fields(nx, ny, nz), steps, probes=probes)
    _, series, _, _ = gpu_run(nx, ny, nz, d, d, d, dt, "fadi", prec, W.zero_fields(nx, ny, nz), steps,
                              eps=eps, source=src, probes=probes)
    for a, b in zip(series, ref):
        assert np.max(np.abs(a - b)) <= TOL[prec] * np.max(np.abs(b)), (np.max(np.abs(a - b)), np.max(np.abs(b)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tuned_per_node_shapes_match_oracle(prec):
    """Per-node handles time their y/z launch shapes at the first step; the
    tuned run (any shape) and every fixed segment length give the oracle's answer."""
    nx, ny, nz = 30, 70, 45
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 6.0 * g.dt_cfl()
    eps = W.eps_blocks(17, nx, ny, nz, 1.0, 6.0)
    u0 = random_fields(nx, ny, nz, seed=17)
    ref, _, _ = S.run_fundamental(S.Problem(g, dt, eps_r_cell=eps), "fss", u0, 5)
    for tune in ((0, 0), (8, 0), (16, 0), (32, 0)):
        out, _, _, _ = gpu_run(nx, ny, nz, d, d, d, dt, "fss", prec, u0, 5, eps=eps, tune=tune)
        check(out, ref, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_flod2_probes_vs_oracle(prec):
    """FLOD2 probe series: the output processing (Eq. 23) of every step's state."""
    nx, ny, nz = 22, 19, 17
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 6.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=31)
    steps = 15
    probes = [("ex", 5, 6, 7), ("hz", 10, 3, 9), ("ez", 1, 1, 1)]
    P = S.Problem(g, dt)
    ref_u, _, ref = S.run_fundamental(P, "flod2", u0, steps, probes=probes)
    out, series, _, _ = gpu_run(nx, ny, nz, d, d, d, dt, "flod2", prec, u0, steps, probes=probes)
    check(out, ref_u, prec)
    for a, b in zip(series, ref):
        assert np.max(np.abs(a - b)) <= TOL[prec] * np.max(np.abs(b))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme,media", [("fadi", "uniform"), ("fss", "blocks"), ("flod", "blocks"),
                                          ("fadi", "blocks+source"), ("fss", "blocks+source"),
                                          ("flod2", "uniform+source")])
def test_graph_steps_bit_identical_to_stream_steps(scheme, media, prec):
    """Steps without probes replay a captured one-step graph whose pairs run
    on parallel branches (a source is read from a device table indexed by a
    device step counter); tune[1] bit 3 forces the stream path.  Same kernels
    and arguments: identical fields; and the oracle's answer."""
    nx, ny, nz = 40, 33, 29
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 5.0 * g.dt_cfl()
    steps = 9
    u0 = random_fields(nx, ny, nz, seed=77)
    eps = W.eps_blocks(77, nx, ny, nz, 1.0, 4.0) if media.startswith("blocks") else None
    src = None
    if media.endswith("source"):
        cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 30) * 1e-4
        src = ("ez", 20, 16, 14, cur)
    a, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, scheme, prec, u0, steps, eps=eps, source=src,
                         tune=(16, 0))
    b, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, scheme, prec, u0, steps, eps=eps, source=src,
                         tune=(16, 8))
    for c in G.COMPS:
        assert np.array_equal(a[c], b[c]), c
    P = oracle_problem(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, eps=eps, source=src)
    ref, _, _ = S.run_fundamental(P, scheme, u0, steps)
    check(a, ref, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_general_media_eps_and_mu_vs_oracle(scheme, prec):
    """Per-cell eps and mu (mu averaged over the two cells of each H face):
    every scheme, ragged grid, a dipole and a probe, against the oracle."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 26, 21, 18
    d = (1e-3, 0.9e-3, 1.2e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 5.0 * g.dt_cfl()
    rng = np.random.default_rng(61)
    eps = rng.uniform(1.0, 5.0, (nz, ny, nx))
    mu = rng.uniform(1.0, 3.0, (nz, ny, nx))
    u0 = random_fields(nx, ny, nz, seed=62)
    steps = 10
    cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 30) * 1e-4
    src = ("ez", 12, 10, 9, cur)
    P = oracle_problem(nx, ny, nz, *d, dt, eps=eps, source=src)
    P = S.Problem(g, dt, eps_r_cell=eps, mu_r_cell=mu, source=P.source)
    probes = [("hy", 7, 8, 5)] if scheme != "flod2" else []
    ref, _, series = S.run_fundamental(P, scheme, u0, steps, probes=probes)
    sim = Simulation(nx, ny, nz, *d, scheme=scheme, precision=prec, dt=dt)
    sim.set_material(eps, mu)
    sim.set_fields(u0)
    sim.set_source(*src)
    pids = [sim.add_probe(*p) for p in probes]
    sim.step(steps)
    out = {c: sim.get_field(c).astype(np.float64) for c in G.COMPS}
    check(out, ref, prec)
    for pid, s_ref in zip(pids, series):
        got = sim.get_probe(pid, steps)
        assert np.max(np.abs(got - s_ref)) <= TOL[prec] * np.max(np.abs(s_ref))
    assert sim.energy()[0] == pytest.approx(I.energy(g, P.mat, ref), rel=TOL[prec])
    sim.close()


def test_general_media_is_rejected_where_not_built():
    """Batches and the reverse pass take uniform mu only; non-uniform mu needs
    lines of at most 256 cells."""
    from paper_2011_14043_gb300 import Batch, FdtdError, Simulation
    mu = np.ones((8, 9, 10))
    mu[2:4, 3:5, 4:6] = 2.0
    a = Simulation(10, 9, 8, 1e-3, scheme="fadi", precision="f32", cfl=3.0)
    a.set_material(None, mu)
    with pytest.raises(FdtdError):
        Batch([a])
    big = Simulation(300, 4, 4, 1e-3, scheme="flod", precision="f32", cfl=3.0)
    with pytest.raises(FdtdError):
        big.set_material(None, np.ones((4, 4, 300)) + np.arange(300) * 1e-3)


@pytest.mark.parametrize("dims", [(3, 1024, 3), (3, 3, 1024), (1024, 3, 3)])
def test_longest_lines_in_inhomogeneous_media(dims):
    """Per-node media at the longest supported lines (32 segments of 32 nodes
    along y or z, 32 nodes per lane along x), with a source, vs the oracle."""
    nx, ny, nz = dims
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 6.0 * g.dt_cfl()
    eps = np.random.default_rng(sum(dims)).uniform(1.0, 5.0, (nz, ny, nx))
    u0 = random_fields(nx, ny, nz, seed=sum(dims) + 1)
    P = oracle_problem(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, eps=eps)
    ref, _, _ = S.run_fundamental(P, "flod", u0, 3)
    for prec in ("f64", "f32"):
        out, _, _, _ = gpu_run(nx, ny, nz, 1e-3, 1e-3, 1e-3, dt, "flod", prec, u0, 3, eps=eps)
        check(out, ref, prec)


@pytest.mark.parametrize("dims,code", [((1025, 4, 4), -1), ((4, 1025, 4), -6), ((4, 4, 1025), -6)])
def test_lines_past_the_limit_are_rejected(dims, code):
    """Lines longer than 1024 cells are refused at creation, as the header
    states: nx > 1024 is an invalid argument, ny or nz > 1024 (more than 32
    segments of 32 nodes) FDTD_ERR_UNSUPPORTED; the library stays usable."""
    from paper_2011_14043_gb300 import FdtdError, Simulation
    with pytest.raises(FdtdError) as e:
        Simulation(*dims, 1e-3, scheme="fadi", precision="f32", cfl=2.0)
    assert e.value.code == code
    sim = Simulation(8, 8, 8, 1e-3, scheme="fadi", precision="f32", cfl=2.0)
    sim.step(2)
    sim.synchronize()
    sim.close()


@pytest.mark.parametrize("media", ["uniform", "blocks"])
@pytest.mark.parametrize("scheme", ["fadi", "flod", "fss", "flod2"])
def test_fp64_sequential_lines_match_segmented_solve(scheme, media):
    """FP64 y and z lines in pairs of at least 32768 lines: one thread per
    line walking the Thomas recurrences against the segmented solve (tune[1]
    bit 10), equal to a few roundings, and against the oracle to 1e-12;
    lines of 130 and 90 cells, node chunks of 8 with a ragged last chunk;
    uniform eps_r (tabulated factors) and eps_r blocks (per-node pivots)."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 400, 130, 90
    d = (1e-3, 0.9e-3, 1.2e-3)
    g = G.Grid(nx, ny, nz, *d)
    dt = 5.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=31)
    eps = np.full((nz, ny, nx), 1.7) if media == "uniform" else W.eps_blocks(5, nx, ny, nz, 1.0, 6.0)
    out = {}
    for tune in ((0, 0), (0, 1024)):
        sim = Simulation(nx, ny, nz, *d, scheme=scheme, precision="f64", dt=dt, tune=tune)
        sim.set_material(eps)
        sim.set_fields(u0)
        sim.step(4)
        out[tune] = {c: sim.get_field(c) for c in G.COMPS}
        sim.close()
    assert energy_norm_rel(out[(0, 0)], out[(0, 1024)]) <= 1e-13
    ref, _, _ = S.run_fundamental(S.Problem(g, dt, eps_r_cell=eps), scheme, u0, 4)
    assert energy_norm_rel(out[(0, 0)], ref) <= 1e-12


@pytest.mark.parametrize("scheme", ["fadi", "fss"])
def test_full_x_lines_without_masks_bit_identical(scheme):
    """FP32 x lines of exactly 32 L cells (here 256 = 32 x 8) in homogeneous
    media run the wall-corrected kernel without end-of-line masks; with
    tune[1] bit 11 they keep the masked kernel: the same arithmetic on every
    node, so the fields agree to the last bit."""
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz = 256, 20, 17
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    dt = 4.0 * g.dt_cfl()
    u0 = random_fields(nx, ny, nz, seed=44)
    out = []
    for tune in ((0, 0), (0, 2048)):
        sim = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision="f32", dt=dt, tune=tune)
        sim.set_fields(u0)
        sim.step(5)
        out.append({c: sim.get_field(c) for c in G.COMPS})
        sim.close()
    for c in G.COMPS:
        assert np.array_equal(out[0][c], out[1][c]), c
