"""The bounds-checked debug build (-DFDTD_BOUNDS) in place of a memory
sanitizer: every line, tile or element range a kernel touches is checked
against its array's extent.  On cases covering every kernel family
(tests/bounds_cases.py) it must report no violation and give the same
arrays as the default build, bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def run_cases(lib_path, out_path, tune_cache):
    # launch shapes tuned by timing are shared through the cache file, so
    # both builds split the lines into the same segments
    env = dict(os.environ, FDTD_LIBRARY=lib_path, FDTD_TUNE_CACHE=str(tune_cache))
    res = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), str(out_path)], env=env,
                         cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    return np.load(out_path)


def test_bounds_checked_build_runs_clean_and_matches(tmp_path):
    from paper_2011_14043_gb300.build import LIB_PATH, build
    build()
    checked = build(bounds=True)
    cache = tmp_path / "tune_cache.txt"
    ref = run_cases(LIB_PATH, tmp_path / "default.npz", cache)
    chk = run_cases(checked, tmp_path / "checked.npz", cache)
    assert sorted(ref.files) == sorted(chk.files)
    assert len(ref.files) > 500
    for k in ref.files:
        assert np.array_equal(ref[k], chk[k]), k
