"""The integer-pipe microbenchmark that gives the alignment kernel's roofline its peak."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_int_peaks_are_measured():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as gn
    p = gn.gn_measure_int_peaks()
    assert p["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    for k in ("add3_ops", "addmax_plain_ops", "dpx_addmax_ops", "dpx_max3_ops", "dpx_bmax_ops"):
        # operations per second over the device: more than a GHz per SM, less than 8 lanes x 4 ops
        # per clock of every integer lane at 3 GHz
        assert math.isfinite(p[k]) and p["sms"] * 1e9 < p[k] < p["sms"] * 128 * 8 * 3e9, (k, p)
