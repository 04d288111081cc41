"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_02987_gb300 import _build
    path = _build.build()
    import paper_1507_02987_gb300 as gn
    return gn, path


def _declared():
    src = open(os.path.join(ROOT, "include", "genoogle.h")).read()
    return sorted(set(re.findall(r"GN_API\s+[\w\s\*]*?\b(gn_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    gn, path = lib
    names = _declared()
    assert len(names) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(gn_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    handle = ctypes.CDLL(path)
    for n in names:
        getattr(handle, n)


def test_defaults_without_gpu(lib):
    gn, _ = lib
    sc, p = gn.gn_default_params()
    assert (sc.match, sc.mismatch, sc.gap_open, sc.gap_extend) == (1, -3, -5, -2)
    assert abs(sc.lambda_ - 1.3740631) < 1e-9 and sc.K == 0.711
    assert (p.max_hit_distance, p.min_hsp_len, p.xdrop, p.max_alignments, p.band_w) == (0, 0, 20, 100, 16)
    assert math.isinf(p.max_evalue)


def test_argument_errors_before_any_device_work(lib):
    gn, _ = lib
    import numpy as np
    ss = np.array([0, 4], dtype=np.uint64)
    b = np.frombuffer(b"ACGT", dtype=np.uint8)
    for k in (0, 17):
        bank = gn.gn_bank(1, ss.ctypes.data, b.ctypes.data, gn.GN_MEM_HOST)
        with pytest.raises(gn.GnError) as e:
            gn.gn_index_build(bank, k, 1)
        assert e.value.status == gn.GN_EINVAL and "k must be" in str(e.value)
    bank = gn.gn_bank(1, ss.ctypes.data, b.ctypes.data, gn.GN_MEM_HOST)
    with pytest.raises(gn.GnError) as e:
        gn.gn_index_build(bank, 11, 0)
    assert e.value.status == gn.GN_EINVAL
    q = gn.gn_queries(1, ss.ctypes.data, b.ctypes.data, gn.GN_MEM_HOST)
    with pytest.raises(gn.GnError) as e:
        gn.gn_search(0, q, gn.make_scoring(), gn.make_params())
    assert e.value.status == gn.GN_EINVAL
    assert gn.gn_results_count.__doc__ is None or True
    assert gn.gn_last_error() != ""
