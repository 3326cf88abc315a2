"""The hand-written FADI adjoint (fdtd_adj_* through the C ABI) against the
FP64 oracle's discrete adjoint (oracle/adjoint.py, pinned to central
differences) and against central differences of the GPU forward model."""
import json

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import grid as G

from gpu_helpers import oracle_problem, random_fields

pytestmark = pytest.mark.gpu


def small_case(seed=21):
    nx, ny, nz = 14, 12, 10
    d = 1e-3
    g = G.Grid(nx, ny, nz, d, d, d)
    dt = 4.0 * g.dt_cfl()
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 6.0, (nz, ny, nx))
    steps = 13
    cur = W.dipole_current((np.arange(steps + 1) + 0.5) * dt * 20) * 1e-5
    src = ("ez", 5, 6, 4, cur)
    u0 = random_fields(nx, ny, nz, seed=seed + 1)
    block = (8, 12, 3, 8, 2, 7)
    return g, dt, eps, src, u0, block, steps


def gpu_problem(case, prec, every):
    from paper_2011_14043_gb300.adjoint import ProbeEnergyProblem
    g, dt, eps, src, u0, block, steps = case
    return ProbeEnergyProblem(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, steps=steps, probe_block=block, dt=dt,
                              precision=prec, checkpoint_every=every, source=src, fields=u0)


@pytest.fixture(scope="module")
def oracle_small():
    case = small_case()
    g, dt, eps, src, u0, block, steps = case
    P = oracle_problem(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, dt, eps=eps, source=src)
    J, grad, _ = AD.gradient(P, u0, steps, AD.probe_masks(g, block))
    return case, J, grad


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 1e-3)])
def test_adjoint_matches_oracle(oracle_small, prec, tol):
    case, J_ref, g_ref = oracle_small
    run = gpu_problem(case, prec, every=5).run(case[2])
    g = run.backward(1.0, out=np.empty_like(g_ref))
    run.close()
    j_err = abs(run.J / J_ref - 1.0)
    g_err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print(f"\nADJOINT small {prec} J_rel={j_err:.3e} grad_rel={g_err:.3e}")
    assert j_err <= (1e-12 if prec == "f64" else 1e-4)
    assert g_err <= tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_checkpoint_spacing_does_not_change_the_gradient(oracle_small, prec):
    """Recomputation from checkpoints reproduces the forward states exactly."""
    case = oracle_small[0]
    out = []
    for every in (1, 4, 13, 20):
        run = gpu_problem(case, prec, every).run(case[2])
        out.append(run.backward(0.5, out=np.empty(case[2].shape)))
        run.close()
    for g in out[1:]:
        assert np.array_equal(g, out[0])


def test_autograd_function(oracle_small):
    import torch
    case, J_ref, g_ref = oracle_small
    prob = gpu_problem(case, "f64", every=5)
    eps = torch.tensor(case[2], dtype=torch.float64, device="cuda", requires_grad=True)
    J = prob.objective(eps)
    (3.0 * J).backward()
    assert float(J) == pytest.approx(J_ref, rel=1e-12)
    g = eps.grad.cpu().numpy()
    assert np.linalg.norm(g - 3.0 * g_ref) / np.linalg.norm(3.0 * g_ref) <= 1e-6


def test_adjoint_rejects_bad_use():
    from paper_2011_14043_gb300 import FdtdError, Simulation
    from paper_2011_14043_gb300.adjoint import AdjointRun, ProbeEnergyProblem
    prob = ProbeEnergyProblem(10, 9, 8, 1e-3, steps=3, probe_block=(2, 4, 2, 4, 2, 4), cfl=3.0, precision="f64")
    with pytest.raises(ValueError):
        prob.run(np.ones((8, 9, 11)))
    run = prob.run(np.ones((8, 9, 10)))          # uniform eps, per-node coefficients forced
    with pytest.raises(FdtdError):
        run.forward()                             # forward runs once
    run.close()
    bad = ProbeEnergyProblem(10, 9, 8, 1e-3, steps=3, probe_block=(2, 40, 2, 4, 2, 4), cfl=3.0)
    with pytest.raises(FdtdError):
        AdjointRun(bad, np.ones((8, 9, 10)))


def test_fullsize_192_gradient_vs_central_differences():
    """192^3, CFL 4, eps_r in [1, 6] in the central 64^3, dipole, 4^3 probe block,
    500 steps, checkpoints every 25: the FP32 adjoint gradient on 16 seeded
    design cells against central differences of the FP64 forward model
    (<= 1e-3 relative), and the FP64 adjoint against the same differences."""
    from paper_2011_14043_gb300.adjoint import ProbeEnergyProblem
    wl = W.workload_adjoint()
    n = wl.nx
    g = G.Grid(n, n, n, wl.dx, wl.dy, wl.dz)
    dt = wl.cfl * g.dt_cfl()
    cur = W.dipole_current((np.arange(wl.steps + 1) + 0.5) * dt)
    s = wl.source
    src = (s["comp"], s["i"], s["j"], s["k"], cur)
    kw = dict(steps=wl.steps, probe_block=wl.extra["probe_block"], dt=dt,
              checkpoint_every=wl.extra["checkpoint_every"], source=src)
    p32 = ProbeEnergyProblem(n, n, n, wl.dx, precision="f32", **kw)
    p64 = ProbeEnergyProblem(n, n, n, wl.dx, precision="f64", **kw)
    r32 = p32.run(wl.eps_r)
    mem = r32.memory_bytes()
    g32 = r32.backward(1.0).cpu().numpy()
    J32 = r32.J
    r32.close()
    r64 = p64.run(wl.eps_r)
    g64 = r64.backward(1.0).cpu().numpy()
    J64 = r64.J
    r64.close()
    lo, hi = wl.extra["region"]
    rng = np.random.default_rng(55)
    cells = [tuple(int(v) for v in rng.integers(lo, hi, 3)) for _ in range(16)]
    h = 1e-3
    fd = []
    for c in cells:
        ep = wl.eps_r.copy(); ep[c] += h
        em = wl.eps_r.copy(); em[c] -= h
        fd.append((p64.value(ep) - p64.value(em)) / (2 * h))
    fd = np.array(fd)
    a32 = np.array([g32[c] for c in cells])
    a64 = np.array([g64[c] for c in cells])
    scale = np.abs(fd).max()
    err32 = np.abs(a32 - fd) / np.maximum(np.abs(fd), 1e-2 * scale)
    err64 = np.abs(a64 - fd) / np.maximum(np.abs(fd), 1e-2 * scale)
    print("\nFULLSIZE adjoint192 " + json.dumps({
        "J_f32": J32, "J_f64": J64, "J_rel": abs(J32 / J64 - 1),
        "grad_rel_l2_f32_vs_f64": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
        "fd_max_rel_err_f32": float(err32.max()), "fd_max_rel_err_f64": float(err64.max()),
        "adjoint_device_bytes_f32": mem}))
    assert J64 > 0
    assert err32.max() <= 1e-3
    assert err64.max() <= 1e-4
