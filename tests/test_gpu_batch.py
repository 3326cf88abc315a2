"""Batched stepping of many independent cavities (the 64-cavity recipe at
reduced sizes): every grid against the FP64 oracle, and, with the batch's
segment length pinned to the handles' own, against the same grid stepped on
its own (the same arithmetic: bit-identical).  Tuned and fixed launch
shapes against the oracle; the tuner's cache file; one persistent launch
per procedure against the graph of launch groups (bit-identical)."""
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


def make_sim(spec, scheme, prec, tune=(0, 0)):
    from paper_2011_14043_gb300 import Simulation
    nx, ny, nz, cfl, eps, u0 = spec
    sim = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision=prec, cfl=cfl, tune=tune)
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
    batch.set_config(y=(16, 16), z=(16, 16), x_pack=0)   # the handles' own segment lengths
    batch.step(4)
    batch.step(steps - 4)            # a second call replays the same graph
    assert batch.launches_per_step() >= 2
    for sp, sim in zip(specs, sims):
        nx, ny, nz, cfl, eps, u0 = sp
        g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
        ref, _, _ = S.run_fundamental(S.Problem(g, sim.dt, eps_r_cell=eps), scheme, u0, steps)
        got = sim.get_fields()
        assert energy_norm_rel(got, ref) <= TOL[prec]
        alone = make_sim(sp, scheme, prec, tune=(16, 0))    # L = 16, no shape tuning
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


def run_against_oracle(specs, scheme, prec, steps, configure):
    from paper_2011_14043_gb300 import Batch
    sims = [make_sim(sp, scheme, prec) for sp in specs]
    batch = Batch(sims)
    configure(batch)
    batch.step(steps)
    cfg = batch.config()
    for sp, sim in zip(specs, sims):
        nx, ny, nz, cfl, eps, u0 = sp
        g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
        ref, _, _ = S.run_fundamental(S.Problem(g, sim.dt, eps_r_cell=eps), scheme, u0, steps)
        assert energy_norm_rel(sim.get_fields(), ref) <= TOL[prec], cfg
    batch.close()
    return cfg


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tuned_batch_matches_oracle(prec):
    specs = small_batch(77, 6)
    cfg = run_against_oracle(specs, "fadi", prec, 7, lambda b: None)
    assert cfg["y"][1] in (8, 16, 32) and cfg["z"][1] in (8, 16, 32)
    assert cfg["x_warps_per_block"] in (4, 8, 16) and cfg["x_pack"] in (0, 1)


@pytest.mark.parametrize("prec,shape,xpack", [("f32", (32, 8), 1), ("f32", (16, 32), 0), ("f32", (32, 16), 1),
                                              ("f64", (8, 32), 0), ("f64", (16, 8), 1), ("f64", (8, 16), 1)])
def test_fixed_batch_shapes_match_oracle(prec, shape, xpack):
    specs = small_batch(91, 5)
    cfg = run_against_oracle(specs, "flod", prec, 6,
                             lambda b: b.set_config(y=shape, z=shape, x_warps_per_block=4, x_pack=xpack))
    assert cfg["y"] == shape and cfg["z"] == shape and cfg["x_pack"] == xpack


def test_tuner_cache_file(tmp_path, monkeypatch):
    from paper_2011_14043_gb300 import Batch, FdtdError
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("FDTD_TUNE_CACHE", str(path))
    specs = small_batch(123, 3)
    sims = [make_sim(sp, "fadi", "f32") for sp in specs]
    b1 = Batch(sims)
    b1.step(1)
    cfg1 = b1.config()
    mode1 = b1.mode()
    b1.close()
    # one line for the shapes, one for the mode chosen with them
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and lines[0].split()[1:] == [str(v) for v in (*cfg1["y"], *cfg1["z"],
                                                                       cfg1["x_warps_per_block"], cfg1["x_pack"])]
    assert "|mode|" in lines[1] and lines[1].split()[1] == ("1" if mode1["mode"] == "persistent" else "0")
    sims2 = [make_sim(sp, "fadi", "f32") for sp in specs]
    b2 = Batch(sims2)
    b2.step(1)
    assert b2.config()["y"] == cfg1["y"] and b2.config()["z"] == cfg1["z"]
    assert b2.mode()["mode"] == mode1["mode"]
    assert len(path.read_text().splitlines()) == 2     # served from the cache
    with pytest.raises(FdtdError):
        b2.set_config(y=(24, 16), z=(16, 16))
    b2.close()


def per_node_specs(seed):
    """Grids with eps_r blocks (per-node media) of uneven sizes: y lines up to
    121 cells and z lines up to 128 (16 segments of 8: 256-thread tiles, the
    largest a persistent block takes), tiles of 2 to 16 segments packed side
    by side, x lines packed by 8, 16 and 32 lanes."""
    rng = np.random.default_rng(seed)
    d = 1e-3
    out = []
    for nx, ny, nz in [(40, 121, 6), (9, 7, 33), (70, 12, 20), (17, 33, 128), (6, 6, 5), (33, 40, 17),
                       (130, 10, 9)]:
        cfl = float(rng.uniform(2.0, 10.0))
        eps = W.eps_blocks(rng, nx, ny, nz, 1.0, 4.0)
        modes = W.random_modes(rng, nx, ny, nz, d, d, d, count=3, mmax=4)
        out.append((nx, ny, nz, cfl, eps, W.mode_sum_fields(modes, nx, ny, nz)))
    return out


def run_mode(specs, scheme, prec, mode, shape, steps):
    from paper_2011_14043_gb300 import Batch
    sims = [make_sim(sp, scheme, prec) for sp in specs]
    b = Batch(sims)
    b.set_config(y=shape, z=shape, x_pack=1)
    b.set_mode(mode)
    b.step(2)
    b.step(steps - 2)  # a second call replays the same graph
    info = b.mode()
    per_step = b.launches_per_step()
    out = [sm.get_fields() for sm in sims]
    b.close()
    for sm in sims:
        sm.close()
    return out, info, per_step


@pytest.mark.parametrize("prec,shape", [("f64", (16, 8)), ("f32", (16, 8)), ("f32", (16, 16))])
@pytest.mark.parametrize("scheme", ["fadi", "fss"])
def test_persistent_batch_matches_launch_groups(scheme, prec, shape):
    """One persistent launch per procedure (work items of every group of
    every grid) against the graph of shape-uniform launches: the same
    arithmetic per line, so the fields agree to the last bit; one launch per
    procedure; the smallest grid against the FP64 oracle."""
    specs = per_node_specs(70)
    steps = 5
    a, ia, na = run_mode(specs, scheme, prec, "launches", shape, steps)
    p, ip, n_p = run_mode(specs, scheme, prec, "persistent", shape, steps)
    assert ia["mode"] == "launches" and ip["mode"] == "persistent"
    assert n_p == (3 if scheme == "fss" else 2) and na > n_p
    for q, (x, y) in enumerate(zip(a, p)):
        for c in G.COMPS:
            assert np.array_equal(x[c], y[c]), (q, c)
    nx, ny, nz, cfl, eps, u0 = specs[4]
    g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
    from paper_2011_14043_gb300 import Simulation
    dt = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision=prec, cfl=cfl).dt
    ref, _, _ = S.run_fundamental(S.Problem(g, dt, eps_r_cell=eps), scheme, u0, steps)
    assert energy_norm_rel(p[4], ref) <= TOL[prec]


def test_batch_mode_tuned_and_persistent_limits():
    """mode "auto" times both modes on the batch's own data and keeps the
    faster; "persistent" on a batch whose x lines are not packed (uniform
    media), or whose lines need tiles of more than 256 threads, is refused
    at the step."""
    from paper_2011_14043_gb300 import Batch, FdtdError
    specs = per_node_specs(71)
    sims = [make_sim(sp, "fadi", "f32") for sp in specs]
    b = Batch(sims)
    b.set_config(y=(16, 8), z=(16, 8), x_pack=1)  # shapes fixed; the mode still tuned
    b.step(2)
    info = b.mode()
    ms = info["tuned_step_ms"]
    assert ms["launches"] > 0 and ms["persistent"] > 0
    assert info["mode"] == ("persistent" if ms["persistent"] < ms["launches"] else "launches")
    b.close()
    for sm in sims:
        sm.close()
    specs = small_batch(72, 4)
    sims = [make_sim(sp, "fadi", "f32") for sp in specs]
    b = Batch(sims)
    b.set_config(y=(16, 16), z=(16, 16), x_pack=0)
    b.set_mode("persistent")
    with pytest.raises(FdtdError) as err:
        b.step(1)
    assert err.value.code == -6
    b.set_mode("launches")
    b.step(1)
    b.close()
    for sm in sims:
        sm.close()
    spec = per_node_specs(73)[0]
    nx, ny, nz, cfl, eps, u0 = spec
    ny = 140  # 18 segments of 8 along y: a 288-thread tile
    spec = (nx, ny, nz, cfl, np.ones((nz, ny, nx)) * 2.0 + (np.arange(nx) % 2), W.zero_fields(nx, ny, nz))
    sims = [make_sim(spec, "fadi", "f32")]
    b = Batch(sims)
    b.set_config(y=(16, 8), z=(16, 8), x_pack=1)
    b.set_mode("persistent")
    with pytest.raises(FdtdError) as err:
        b.step(1)
    assert err.value.code == -6
    b.close()
    sims[0].close()
