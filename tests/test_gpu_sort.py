"""The library's LSD radix sort (both forms: single-pass passes with decoupled look-back,
and the three-kernel passes that larger sorts take) against numpy's stable sort of the
same digits, and the single-pass form's bounded wait.

A sort by bits [lo, hi) is a stable sort by (key >> lo) & (2^(hi - lo) - 1): keys whose
digits agree keep their input order, and values move with their keys."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as gn
    return gn


def _keys(kind, n, rng):
    if kind == "random":
        return rng.integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True)
    if kind == "few":  # a handful of distinct digits: long runs of equal keys in every tile
        return rng.integers(0, 4, n, dtype=np.uint64) * np.uint64(0x0101010101010101)
    if kind == "equal":
        return np.full(n, 0x123456789ABCDEF0, dtype=np.uint64)
    # record-sort shape: (query, sequence, position) fields packed low, high bits zero
    q = rng.integers(0, 2000, n, dtype=np.uint64)
    s = rng.integers(0, 1 << 22, n, dtype=np.uint64)
    p = rng.integers(0, 1 << 16, n, dtype=np.uint64)
    return (q << np.uint64(38)) | (s << np.uint64(16)) | p


def _run(gn, keys, vals, lo, hi, **kw):
    import torch
    dk = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda() if vals is not None else None
    gn.gn_debug_sort(dk.data_ptr(), dv.data_ptr() if dv is not None else None, len(keys), lo, hi,
                     stream=torch.cuda.current_stream().cuda_stream, **kw)
    return dk.cpu().numpy().view(np.uint64), (dv.cpu().numpy().view(np.uint32) if dv is not None else None)


def _expected(keys, vals, lo, hi):
    width = hi - lo
    mask = np.uint64((1 << width) - 1) if width < 64 else np.uint64(np.iinfo(np.uint64).max)
    digits = (keys >> np.uint64(lo)) & mask if lo < 64 else np.zeros_like(keys)
    perm = np.argsort(digits, kind="stable")
    return keys[perm], (vals[perm] if vals is not None else None)


@pytest.mark.parametrize("three_kernel", [False, True])
@pytest.mark.parametrize("n", [2, 4095, 4096, 4097, 100_003, 1_000_000])
@pytest.mark.parametrize("kind", ["random", "records", "few"])
def test_sort_matches_stable_numpy(gn, three_kernel, n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    keys = _keys(kind, n, rng)
    vals = np.arange(n, dtype=np.uint32)
    for lo, hi in ((0, 64), (16, 60), (5, 37), (32, 48)):
        got_k, got_v = _run(gn, keys, vals, lo, hi, three_kernel=three_kernel)
        exp_k, exp_v = _expected(keys, vals, lo, hi)
        assert np.array_equal(got_k, exp_k), (lo, hi)
        assert np.array_equal(got_v, exp_v), (lo, hi)


@pytest.mark.parametrize("three_kernel", [False, True])
def test_sort_keys_only_and_degenerate(gn, three_kernel):
    rng = np.random.default_rng(3)
    for kind, n in (("equal", 50_000), ("random", 300_000), ("records", 1)):
        keys = _keys(kind, n, rng)
        got_k, _ = _run(gn, keys, None, 0, 64, three_kernel=three_kernel)
        assert np.array_equal(got_k, np.sort(keys, kind="stable")), kind
    keys = _keys("random", 10_000, rng)
    got_k, _ = _run(gn, keys, None, 20, 20, three_kernel=three_kernel)  # no bits: unchanged
    assert np.array_equal(got_k, keys)


def test_sort_wait_runs_out_and_the_device_stays_usable(gn):
    """The first tile never publishes its digit counts: every later tile's look-back runs
    out after its bound (GN_ETIMEOUT), and the next sort is right."""
    import torch
    rng = np.random.default_rng(5)
    keys = _keys("random", 4096 * 40, rng)
    vals = np.arange(len(keys), dtype=np.uint32)
    with pytest.raises(gn.GnError) as e:
        _run(gn, keys, vals, 0, 16, wait_cycles=2_000_000, drop_first=True)
    assert e.value.status == gn.GN_ETIMEOUT
    got_k, got_v = _run(gn, keys, vals, 0, 16)
    exp_k, exp_v = _expected(keys, vals, 0, 16)
    assert np.array_equal(got_k, exp_k) and np.array_equal(got_v, exp_v)
    torch.cuda.synchronize()
