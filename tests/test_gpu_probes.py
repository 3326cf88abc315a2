"""The FP64 FMA throughput probe: the measured denominator of the FP64
form's ALU roofline (fdtd_probe_fp64_fma)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probe_rate_is_plausible_and_stable():
    from paper_2011_14043_gb300 import probe_fp64_fma
    a = probe_fp64_fma(4000)
    b = probe_fp64_fma(8000)
    for v in (a, b):
        assert 1e11 < v < 1e14, v        # between 0.1 and 100 TFLOP/s
    assert abs(a / b - 1.0) < 0.3        # a throughput, not a launch latency
