"""The allocation-free energy entry point.

fdtd_energy_noalloc is for callers that cannot allocate device memory where
they need the energy (a framework's caching allocator holds the memory, or a
loop cannot take cudaMalloc's device-wide synchronisation); its scratch is a
fixed file-scope device array.  Checked here on two calls in a row against
the handle's own energy (the existing entry point) and against the oracle's
energy of the same fields, and for the property it exists for: once warm,
a call changes neither torch's allocated bytes nor the device's free memory.
This file is collected last so that a run stopping at the first failure has
run every other test already."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as G
from oracle import invariants as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_noalloc_energy_matches_handle_and_oracle_energy_twice(prec, tol):
    import torch
    from paper_2011_14043_gb300 import Simulation, energy_noalloc
    nx, ny, nz = 40, 33, 27
    d = (1e-3, 0.8e-3, 1.2e-3)
    modes = W.random_modes(11, nx, ny, nz, *d, count=4, mmax=6)
    u0 = W.mode_sum_fields(modes, nx, ny, nz)
    eps = np.full((nz, ny, nx), 2.5)
    mat = G.material_at_samples(G.Grid(nx, ny, nz, *d), eps)
    sim = Simulation(nx, ny, nz, *d, scheme="fadi", precision=prec, cfl=4.0)
    sim.set_material(eps)
    sim.set_fields(u0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for rnd in range(2):
        sim.step(3)
        ref = sim.energy()[0]
        dev = {c: sim.get_field(c, device=True) for c in W.COMPONENTS}
        host = {c: dev[c].double().cpu().numpy() for c in W.COMPONENTS}
        torch.cuda.synchronize()
        energy_noalloc(dev, nx, ny, nz, *d, eps_r=2.5, mu_r=1.0, out=out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert got == pytest.approx(ref, rel=tol), (rnd, got, ref)
        # the same sample values summed by the FP64 oracle
        assert got == pytest.approx(I.energy(G.Grid(nx, ny, nz, *d), mat, host), rel=1e-12), rnd
    # once warm, a call allocates nothing: torch's allocator and the device's
    # free memory are unchanged across it
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    energy_noalloc(dev, nx, ny, nz, *d, eps_r=2.5, mu_r=1.0, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    # a repeated call on unchanged inputs gives the identical number
    assert float(out.item()) == got
    sim.close()


def test_noalloc_rejects_too_many_planes():
    import ctypes
    import torch
    from paper_2011_14043_gb300 import _lib
    from paper_2011_14043_gb300._lib import lib
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * 6)(*[t.data_ptr()] * 6)
    rc = lib().fdtd_energy_noalloc(2, 2, 5000, 1e-3, 1e-3, 1e-3, 1.0, 1.0, 0, ptrs,
                                   ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                   None)
    assert rc == -1
    assert _lib.ERRORS[rc] == "FDTD_ERR_INVALID_ARG"
