"""Parity at full size for the two workloads the per-config tests leave out: the 4 Gbp
bank indexed at stride 1, and the serving workload (Poisson arrivals of the serving
request mix against the resident 4 Gbp index).

The oracle side uses an index restricted to the sampled queries' seed codes, whose
buckets equal the full index's (pinned on the CPU in tests/test_oracle_index.py): the
full oracle index at stride 1 would need about 32 GB of host memory and ten minutes to
build.  Host memory used: the 4.0 Gbp bank (4 GB) and the restricted index (under 1 GB
at stride 1)."""
import os
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
          ("score", "score"), ("rank", "rank"))


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
def large_bank():
    return synth.make_bank("large")


def check_with_oracle(bank, qs, got, stride):
    """got[j]: the GPU's ranked alignments of qs.query(j); compared with the oracle."""
    ox = oracle.Index(bank, k=11, stride=stride, restrict_to=qs, threads=os.cpu_count() or 1)
    ref = ox.search(qs, oracle.Params(stride=stride), threads=os.cpu_count() or 1)
    n = 0
    for j in range(qs.n):
        g, e = got[j], ref[j].ranked
        assert len(g) == len(e), f"query {j}: {len(g)} vs {len(e)} alignments"
        for fg, fe in FIELDS:
            assert np.array_equal(g[fg].astype(np.int64), e[fe].astype(np.int64)), f"query {j} field {fg}"
        tiny = (np.abs(g["evalue"]) < 1e-300) & (np.abs(e["evalue"]) < 1e-300)
        assert (tiny | np.isclose(g["evalue"], e["evalue"], rtol=1e-9, atol=0)).all(), f"query {j} evalue"
        n += len(g)
    return n


def same(a, b):
    if len(a) != len(b):
        return False
    if not all(np.array_equal(a[f], b[f]) for f, _ in FIELDS):
        return False
    tiny = (np.abs(a["evalue"]) < 1e-300) & (np.abs(b["evalue"]) < 1e-300)
    return bool((tiny | np.isclose(a["evalue"], b["evalue"], rtol=1e-9, atol=0)).all())


def test_large_config_stride1_sampled(gn, large_bank):
    """The large workload (2,000 queries, one gn_search) against the 4 Gbp bank indexed at
    stride 1 (about 4.0 G occurrences, 8.7 G hits: the fill keeps about half of them, spills
    and re-plans); 20 evenly spaced queries and the last one against the oracle."""
    qs = synth.make_queries("large", large_bank)
    ix = gn.Index.from_bank(large_bank, k=11, stride=1)
    res = gn.search(ix, qs.start, qs.bases)
    idx = list(range(0, qs.n, qs.n // 20))[:20] + [qs.n - 1]
    got = [res.query(i).copy() for i in idx]
    res.close()
    ix.close()
    assert check_with_oracle(large_bank, qs.subset(idx), got, stride=1) > 200


def test_serving_full_size(gn, large_bank):
    """The serving workload: requests of the serving recipe (log-uniform 50-20,000 bp, 30 %
    planted homologs) arrive as a Poisson stream at 2,000 requests/s, then in one burst, at
    the request loop over the resident 4 Gbp index (stride 11, 16 GiB budget).  Every served
    result equals a lone gn_search of the same request, and a sample equals the oracle."""
    spec = synth.QUERIES["serving"]
    qs = synth.make_queries(spec, large_bank)
    n_stream, n_burst = 600, 400
    reqs = [qs.query(i) for i in range(n_stream + n_burst)]
    arrivals = np.concatenate([synth.poisson_arrivals(2000.0, n_stream, seed=spec.seed + 2000),
                               np.zeros(n_burst)])
    arrivals[n_stream:] = arrivals[n_stream - 1]
    ix = gn.Index.from_bank(large_bank, k=11, stride=11)
    srv = gn.Server(ix, 16 << 30)
    t0 = time.perf_counter()
    tickets = []
    for i, q in enumerate(reqs):
        wait = t0 + float(arrivals[i]) - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(q))
    served = {}
    while len(served) < len(reqs):
        got = srv.poll_any(60000)
        assert got is not None, "a request did not finish within 60 s"
        t, res = got
        served[t] = res.query(0).copy()
        res.close()
    stats = srv.stats()
    srv.stop()
    assert stats["max_batch"] > 1 and stats["max_concurrent"] > 1  # batched, overlapping on the device
    mism = []
    for i, q in enumerate(reqs):
        one = synth.queries_from_strings([q])
        r = gn.search(ix, one.start, one.bases)
        if not same(served[tickets[i]], r.query(0)):
            mism.append(i)
        r.close()
    ix.close()
    assert not mism, f"{len(mism)} served results differ from the lone search, e.g. request {mism[:5]}"
    idx = list(range(0, len(reqs), len(reqs) // 30))[:30]
    sample = qs.subset(idx)
    assert check_with_oracle(large_bank, sample, [served[tickets[i]] for i in idx], stride=11) > 50
