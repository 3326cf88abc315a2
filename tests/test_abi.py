"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/fdtd.h declares; argument validation happens before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2011_14043_gb300 import build, _lib
    build()
    return _lib.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z_0-9]+)\s*\(", src)))


def test_header_lists_the_calls():
    names = header_functions()
    assert "fdtd_create" in names and "fdtd_step" in names and "fdtd_energy" in names


def test_library_exports_every_declared_symbol(L):
    from paper_2011_14043_gb300 import _lib
    for name in header_functions():
        assert hasattr(L, name), name
    assert set(header_functions()) == set(_lib.EXPORTS)


def test_desc_struct_layout_matches_header(L):
    from paper_2011_14043_gb300._lib import FdtdDesc
    # 3 int32, pad to 8, 5 doubles, 2 int32 scheme/precision, 2 int32 tune
    assert ctypes.sizeof(FdtdDesc) == 16 + 40 + 8 + 8


def make_desc(**kw):
    from paper_2011_14043_gb300._lib import FdtdDesc
    d = FdtdDesc()
    d.nx, d.ny, d.nz = kw.get("n", (8, 8, 8))
    d.dx = d.dy = d.dz = kw.get("dx", 1e-3)
    d.dt = kw.get("dt", 0.0)
    d.cfl = kw.get("cfl", 4.0)
    d.scheme = kw.get("scheme", 0)
    d.precision = kw.get("precision", 1)
    return d


@pytest.mark.parametrize("bad", [
    dict(n=(1, 8, 8)), dict(n=(8, 0, 8)), dict(n=(8, 8, 0)), dict(dx=0.0), dict(dx=-1.0),
    dict(dx=float("nan")), dict(cfl=0.0, dt=0.0), dict(cfl=float("inf")), dict(scheme=7),
    dict(precision=5), dict(n=(2048, 8, 8)),
])
def test_create_rejects_bad_descriptors(L, bad):
    d = make_desc(**bad)
    h = ctypes.c_void_p()
    rc = L.fdtd_create(ctypes.byref(d), None, ctypes.byref(h))
    assert rc == -1
    assert not h.value


def test_null_handle_and_pointers(L):
    assert L.fdtd_create(None, None, None) == -1
    assert L.fdtd_step(None, 1) == -1
    assert L.fdtd_energy(None, None) == -1
    assert L.fdtd_destroy(None) == 0
    assert L.fdtd_get_field(None, 0, None, 0) == -1
    assert L.fdtd_strerror(-3).decode().startswith("CUDA error")
    assert L.fdtd_strerror(12345).decode() == "unknown error"


@pytest.mark.parametrize("limit", [0, -5, 10_000_000_001])
def test_bounded_wait_selftest_rejects_bad_limits(L, limit):
    assert L.fdtd_selftest_bounded_wait(limit, 0, None) == -1


@pytest.mark.parametrize("iters", [0, -1, 1_000_001])
def test_fp64_probe_rejects_bad_arguments(L, iters):
    v = ctypes.c_double()
    assert L.fdtd_probe_fp64_fma(iters, ctypes.byref(v), None) == -1
    assert L.fdtd_probe_fp64_fma(10, None, None) == -1


def test_energy_noalloc_binding_checks_before_launching(monkeypatch):
    """The Python face of fdtd_energy_noalloc validates every tensor before
    anything reaches the library: an `out` on the host or of another dtype,
    or fields that are not CUDA tensors, raise ValueError (the library is
    replaced by a stub that fails the test if called)."""
    import torch
    import paper_2011_14043_gb300 as P

    def no_call():
        raise AssertionError("the library must not be reached")

    monkeypatch.setattr(P, "lib", no_call)
    nx, ny, nz = 3, 4, 5
    fields = {c: torch.zeros(P.comp_shape(c, nx, ny, nz), dtype=torch.float64) for c in P.COMPS}
    with pytest.raises(ValueError, match="out"):
        P.energy_noalloc(fields, nx, ny, nz, 1e-3, 1e-3, 1e-3, out=torch.zeros(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="out"):
        P.energy_noalloc(fields, nx, ny, nz, 1e-3, 1e-3, 1e-3, out=torch.zeros(1, dtype=torch.float32))
    with pytest.raises(ValueError, match="out"):
        P.energy_noalloc(fields, nx, ny, nz, 1e-3, 1e-3, 1e-3, out=torch.zeros(0, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        P.energy_noalloc(fields, nx, ny, nz, 1e-3, 1e-3, 1e-3)
    mixed = dict(fields)
    mixed["hz"] = mixed["hz"].float()
    with pytest.raises(ValueError, match="dtype"):
        P.energy_noalloc(mixed, nx, ny, nz, 1e-3, 1e-3, 1e-3)
