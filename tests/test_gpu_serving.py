"""The request loop (gn_serve_*): continuous batching over a resident index.

Each query's result must be the same whether it runs alone (one gn_search of
that query) or inside the server's micro-batches, mixed with other requests
that arrive while earlier batches are still on the device.  Admission by
memory footprint, the completion queue and the error paths are checked too."""
import threading
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ["seq", "q_start", "q_end", "db_start", "db_end", "score", "rank"]


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="module")
def served(gn):
    bank = synth.make_bank("mid", n_seqs=20000)
    q1 = synth.make_queries("mid", bank, n=60)
    q2 = synth.make_queries("batched", bank, n=60)
    queries = [q1.query(i) for i in range(q1.n)] + [q2.query(i) for i in range(q2.n)]
    ix = gn.Index.from_bank(bank)
    alone = []
    for q in queries:
        one = synth.queries_from_strings([q])
        alone.append(gn.search(ix, one.start, one.bases).query(0))
    return bank, ix, queries, alone


def same(a, b):
    if len(a) != len(b):
        return False
    if not all(np.array_equal(a[f], b[f]) for f in FIELDS):
        return False
    tiny = (np.abs(a["evalue"]) < 1e-300) & (np.abs(b["evalue"]) < 1e-300)
    return bool((tiny | np.isclose(a["evalue"], b["evalue"], rtol=1e-9, atol=0)).all())


def run_mix(gn, ix, queries, budget, threads=3, gap_s=0.0005):
    """Submits every query from `threads` client threads (interleaved order, short gaps) and
    collects the results through the completion queue; returns ({query index: result}, stats)."""
    srv = gn.Server(ix, budget)
    tickets = {}
    lock = threading.Lock()

    def client(part):
        for i in part:
            t = srv.submit(queries[i])
            with lock:
                tickets[t] = i
            time.sleep(gap_s)

    order = list(range(len(queries)))
    np.random.default_rng(3).shuffle(order)
    ths = [threading.Thread(target=client, args=(order[j::threads],)) for j in range(threads)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    out = {}
    while len(out) < len(queries):
        got = srv.poll_any(60000)
        assert got is not None, "a request did not finish within 60 s"
        t, res = got
        assert res.n_queries == 1
        out[tickets[t]] = res.query(0)
        res.close()
    stats = srv.stats()
    srv.stop()
    return out, stats


def test_each_result_same_alone_and_in_the_mix(gn, served):
    bank, ix, queries, alone = served
    # room for three micro-batches of a few queries each (16 MiB fixed per batch), so
    # batches queue up and overlap
    budget = 3 * (16 << 20) + (3 << 20)
    for attempt in range(3):
        got, stats = run_mix(gn, ix, queries, budget)
        for i, r in got.items():
            assert same(r, alone[i]), f"query {i} differs in the mix"
        assert stats["requests"] == len(queries)
        assert stats["batches"] > 1 and stats["peak_in_use"] <= budget
        if stats["max_concurrent"] >= 2:
            break
    assert stats["max_concurrent"] >= 2, stats  # micro-batches were in flight together
    assert sum(len(r) for r in alone) > 100


def test_large_budget_batches_many(gn, served):
    bank, ix, queries, alone = served
    got, stats = run_mix(gn, ix, queries, 4 << 30, threads=1, gap_s=0.0)
    assert all(same(got[i], alone[i]) for i in range(len(queries)))
    assert stats["max_batch"] > 1


def test_poll_by_ticket(gn, served):
    bank, ix, queries, alone = served
    srv = gn.Server(ix, 1 << 30)
    ts = [srv.submit(queries[i]) for i in range(5)]
    for i, t in reversed(list(enumerate(ts))):
        r = srv.poll(t, 60000)
        assert r is not None and same(r.query(0), alone[i])
        r.close()
    assert srv.poll(ts[0] + 1000, 10) is None  # never submitted: times out
    assert srv.poll_any(10) is None
    srv.stop()


def test_admission_limits(gn, served):
    bank, ix, queries, alone = served
    with pytest.raises(gn.GnError) as e:
        gn.Server(ix, 16 << 20)
    assert e.value.status == gn.GN_EINVAL
    srv = gn.Server(ix, (16 << 20) + (1 << 20))
    # 60,000 bases: 3.84 MB of per-offset arrays alone; submit only queues it, and the
    # ticket fails with GN_ETOOBIG once its footprint is known
    big = srv.submit(b"ACGT" * 15000)
    with pytest.raises(gn.GnError) as e:
        srv.poll(big, 60000)
    assert e.value.status == gn.GN_ETOOBIG
    with pytest.raises(gn.GnError) as e:
        srv.submit(b"A" * 70000)
    assert e.value.status == gn.GN_ETOOBIG
    t = srv.submit(queries[0][:200])
    r = srv.poll(t, 60000)
    one = synth.queries_from_strings([queries[0][:200]])
    assert same(r.query(0), gn.search(ix, one.start, one.bases).query(0))
    r.close()
    t = srv.submit(b"")
    r = srv.poll(t, 60000)
    assert r.n_queries == 1 and len(r.query(0)) == 0
    r.close()
    srv.stop()
