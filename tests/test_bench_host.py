"""CPU checks of bench.py's host-side bookkeeping: the committed DRAM record is
used only for the grid and the kernel sources it was captured with, and the
error norm of the stated FP32 error is the vacuum energy norm."""
import json
import math
import os

import numpy as np
import pytest

import bench


def test_traffic_record_is_used_only_while_current():
    """While the record's key matches the kernel sources, its figures are
    reported and are self-consistent; once the sources change, none is."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")))
    assert rec["grid"] == 256
    current = rec["sources_sha1"] == bench.kernel_sources_sha1()
    for cls in ("y-lines", "z-lines", "x-lines"):
        v = bench.recorded_traffic(cls, 256)
        c = rec["classes"][cls]
        assert c["traffic_bytes_per_launch"] == c["dram_bytes_read"] + c["dram_bytes_write"]
        # reads are the pair's algorithmic reads (E and H, 2 x 256^3 x 4 B), within 1 %
        assert abs(c["dram_bytes_read"] / (2 * 256 ** 3 * 4) - 1) < 0.01
        assert v == (c["traffic_bytes_per_launch"] if current else None)


def test_traffic_record_is_not_used_for_another_grid_or_changed_sources(monkeypatch):
    assert bench.recorded_traffic("x-lines", 192) is None
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda: "0" * 40)
    assert bench.recorded_traffic("x-lines", 256) is None


def test_error_norm_is_the_vacuum_energy_norm():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    comps = ("ex", "ey", "ez", "hx", "hy", "hz")
    b = {c: torch.tensor(rng.standard_normal((3, 4, 5))) for c in comps}
    a = {c: b[c] + 1e-3 * torch.tensor(rng.standard_normal((3, 4, 5))) for c in comps}
    mu0 = 1.25663706212e-6
    eps0 = 1.0 / (mu0 * 299792458.0 ** 2)
    num = sum((eps0 if c[0] == "e" else mu0) * float(((a[c] - b[c]) ** 2).sum()) for c in comps)
    den = sum((eps0 if c[0] == "e" else mu0) * float((b[c] ** 2).sum()) for c in comps)
    assert bench.device_rel_err(a, b) == pytest.approx(math.sqrt(num / den), rel=1e-12)
    # the same offset on every E sample or on every H sample: the errors differ
    # by the vacuum impedance, sqrt(mu0 / eps0) = c0 mu0
    a_e = {c: (b[c] + 1.0 if c[0] == "e" else b[c]) for c in comps}
    a_h = {c: (b[c] + 1.0 if c[0] == "h" else b[c]) for c in comps}
    ratio = bench.device_rel_err(a_h, b) / bench.device_rel_err(a_e, b)
    assert ratio == pytest.approx(299792458.0 * mu0, rel=1e-9)
