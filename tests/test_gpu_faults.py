"""Error paths under injected device-allocation failures (no GPU fault is involved: the
library's allocator reports an out-of-memory error as the device would).

Every allocation a search makes is failed once in turn: the call must return GN_ENOMEM,
hold no device allocation afterwards, and the next search must give the same results.
A micro-batch of the request loop whose allocation fails fails its tickets with
GN_ENOMEM, and the server keeps serving."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("query", "seq", "q_start", "q_end", "db_start", "db_end", "score", "rank")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as gn
    bank = synth.make_bank("mid", n_seqs=3000)
    qs = synth.make_queries("mid", bank, n=20)
    ix = gn.Index.from_bank(bank)
    yield gn, ix, qs
    gn.gn_debug_fail_alloc(0)
    ix.close()


def _all(res):
    out = res.all()
    res.close()
    return out


def _same(a, b):
    return len(a) == len(b) and all(
        len(x) == len(y) and all(np.array_equal(x[f], y[f]) for f in FIELDS if f in x.dtype.names)
        for x, y in zip(a, b))


def test_each_search_allocation_failure_is_clean(env):
    gn, ix, qs = env
    ref = _all(gn.search(ix, qs.start, qs.bases))
    c0 = gn.gn_debug_alloc_count()
    _all(gn.search(ix, qs.start, qs.bases))
    n_alloc = gn.gn_debug_alloc_count() - c0
    assert n_alloc >= 10
    assert gn.gn_debug_live_allocs() == 0
    for nth in range(1, n_alloc + 1):
        gn.gn_debug_fail_alloc(nth)
        with pytest.raises(gn.GnError) as e:
            gn.search(ix, qs.start, qs.bases)
        gn.gn_debug_fail_alloc(0)
        assert e.value.status == gn.GN_ENOMEM, (nth, e.value)
        assert gn.gn_debug_live_allocs() == 0, nth  # everything the failed call held is freed
    assert _same(_all(gn.search(ix, qs.start, qs.bases)), ref)


def test_serving_batch_allocation_failure(env):
    gn, ix, qs = env
    queries = [qs.query(i) for i in range(qs.n)]
    alone = []
    for q in queries:
        one = synth.queries_from_strings([q])
        alone.append(_all(gn.search(ix, one.start, one.bases))[0])
    srv = gn.Server(ix, 1 << 30)
    # the next micro-batch's first allocation fails: each of its tickets reports GN_ENOMEM
    gn.gn_debug_fail_alloc(1)
    ts = [srv.submit(q) for q in queries[:8]]
    failed = ok = 0
    for i, t in enumerate(ts):
        try:
            r = srv.poll(t, 60000)
        except gn.GnError as e:
            assert e.status == gn.GN_ENOMEM, e
            failed += 1
            continue
        assert r is not None
        got = r.query(0)
        assert len(got) == len(alone[i]) and all(np.array_equal(got[f], alone[i][f]) for f in FIELDS[1:])
        r.close()
        ok += 1
    gn.gn_debug_fail_alloc(0)
    assert failed >= 1 and failed + ok == 8
    # the server keeps serving, with identical results
    ts = [srv.submit(q) for q in queries]
    for i, t in enumerate(ts):
        r = srv.poll(t, 60000)
        got = r.query(0)
        assert len(got) == len(alone[i]) and all(np.array_equal(got[f], alone[i][f]) for f in FIELDS[1:])
        r.close()
    srv.stop()
    assert gn.gn_debug_live_allocs() == 0


@pytest.mark.parametrize("n", [1, 4096, 4097, 2048 * 5 + 3, 1_000_003])
def test_single_pass_scan(env, n):
    """The single-pass scan (decoupled look-back) against numpy's cumulative sum."""
    gn, ix, qs = env
    import torch
    rng = np.random.default_rng(n)
    a = rng.integers(0, 1 << 20, n, dtype=np.uint32)
    din = torch.from_numpy(a.view(np.int32)).cuda()
    dout = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    gn.gn_debug_scan(din.data_ptr(), dout.data_ptr(), n, stream=torch.cuda.current_stream().cuda_stream)
    exp = np.concatenate([[0], np.cumsum(a, dtype=np.uint64)])
    assert np.array_equal(dout.cpu().numpy().view(np.uint64), exp)


def test_scan_wait_runs_out_and_the_device_stays_usable(env):
    """A wait that nothing ends (the first tile never publishes its sum) runs out after its
    bound: GN_ETIMEOUT, and the next scan and search work."""
    gn, ix, qs = env
    import torch
    n = 2048 * 64
    a = np.ones(n, dtype=np.uint32)
    din = torch.from_numpy(a.view(np.int32)).cuda()
    dout = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    sh = torch.cuda.current_stream().cuda_stream
    with pytest.raises(gn.GnError) as e:
        gn.gn_debug_scan(din.data_ptr(), dout.data_ptr(), n, wait_cycles=2_000_000, drop_first=True, stream=sh)
    assert e.value.status == gn.GN_ETIMEOUT
    gn.gn_debug_scan(din.data_ptr(), dout.data_ptr(), n, stream=sh)
    assert np.array_equal(dout.cpu().numpy(), np.arange(n + 1))
    ref = _all(gn.search(ix, qs.start, qs.bases))
    assert len(ref) == qs.n
