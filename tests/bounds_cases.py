"""Cases run through one build of the library (the one FDTD_LIBRARY names,
else the default build), saved to an .npz: the bounds-checked build must run
them without a bounds error and give the same arrays as the default build
(tests/test_gpu_bounds.py).  Covers every kernel family: the TMA-fed and
direct y/z kernels, the x-line kernels, per-node and general media, the FADI
initialization and output transforms, sources and probes, graph and stream
paths, batches and the adjoint."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import workloads as W  # noqa: E402
from gpu_helpers import COMPS, random_fields  # noqa: E402
from oracle import grid as G  # noqa: E402


def main(out_path):
    from paper_2011_14043_gb300 import Batch, Simulation
    from paper_2011_14043_gb300.adjoint import ProbeEnergyProblem
    out = {}

    def save(tag, sim):
        sim.synchronize()  # raises FdtdError (FDTD_ERR_BOUNDS) after a bounds violation
        for c in COMPS:
            out[f"{tag}/{c}"] = sim.get_field(c)
        out[f"{tag}/energy"] = np.array(sim.energy())

    dims_list = [(37, 29, 23), (20, 256, 7), (256, 12, 9), (5, 4, 3)]
    for prec in ("f32", "f64"):
        for dims in dims_list:
            nx, ny, nz = dims
            g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
            u0 = random_fields(nx, ny, nz, seed=nx + ny + nz)
            for scheme in ("fadi", "flod", "fss", "flod2"):
                for media in ("uniform", "blocks", "general"):
                    for path in (0, 8):
                        tag = f"{prec}/{nx}x{ny}x{nz}/{scheme}/{media}/{path}"
                        sim = Simulation(nx, ny, nz, 1e-3, scheme=scheme, precision=prec, cfl=5.0, tune=(0, path))
                        if media == "blocks":
                            sim.set_material(W.eps_blocks(7, nx, ny, nz, 1.0, 4.0))
                        elif media == "general" and max(dims) <= 256:
                            rng = np.random.default_rng(3)
                            sim.set_material(rng.uniform(1.0, 4.0, (nz, ny, nx)), rng.uniform(1.0, 3.0, (nz, ny, nx)))
                        sim.set_fields(u0)
                        if media != "uniform":
                            cur = W.dipole_current((np.arange(5) + 0.5) * sim.dt * 30) * 1e-4
                            sim.set_source("ez", nx // 2, ny // 2, nz // 2, cur)
                            pid = sim.add_probe("ez", nx // 2, ny // 2, max(nz // 2 - 1, 0))
                        sim.step(4)
                        if media != "uniform":
                            out[tag + "/probe"] = sim.get_probe(pid, 4)
                        save(tag, sim)
                        sim.close()
        # a batch of three grids, uniform and per-node media
        sims = []
        for q, (nx, ny, nz) in enumerate([(33, 20, 17), (48, 40, 12), (20, 31, 26)]):
            sim = Simulation(nx, ny, nz, 1e-3, scheme="fadi", precision=prec, cfl=4.0)
            if q == 1:
                sim.set_material(W.eps_blocks(5, nx, ny, nz, 1.0, 4.0))
            sim.set_fields(random_fields(nx, ny, nz, seed=40 + q))
            sims.append(sim)
        b = Batch(sims)
        b.step(5)
        b.synchronize()
        for q, sim in enumerate(sims):
            save(f"{prec}/batch/{q}", sim)
        b.close()
        for sim in sims:
            sim.close()
        # the adjoint (checkpointed forward, recomputation, reverse pass)
        nx, ny, nz = 14, 12, 10
        g = G.Grid(nx, ny, nz, 1e-3, 1e-3, 1e-3)
        dt = 4.0 * g.dt_cfl()
        cur = W.dipole_current((np.arange(9) + 0.5) * dt * 20) * 1e-5
        prob = ProbeEnergyProblem(nx, ny, nz, 1e-3, steps=8, probe_block=(8, 12, 3, 8, 2, 7), dt=dt,
                                  precision=prec, checkpoint_every=3, source=("ez", 5, 6, 4, cur),
                                  fields=random_fields(nx, ny, nz, seed=9))
        eps = np.random.default_rng(4).uniform(1.0, 6.0, (nz, ny, nx))
        run = prob.run(eps)
        out[f"{prec}/adjoint/J"] = np.array([run.J])
        out[f"{prec}/adjoint/grad"] = run.backward(1.0, out=np.empty((nz, ny, nx)))
        run.close()
    np.savez(out_path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
