"""Parity at the full workload sizes, in the launch configuration the benchmark times.

Each test builds the full synthetic bank, searches the whole query set in one
gn_search call (as bench.py does), and compares evenly spaced sampled queries
with the oracle, which searches those queries alone.  The per-query result of
the method does not depend on the other queries of the batch, so the sampled
comparison is exact: integers identical, e-values within 1e-9 relative."""
import os

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


def compare_sampled(gn, bank, qs, n_sample, stride=11):
    ix = gn.Index.from_bank(bank, k=11, stride=stride)
    res = gn.search(ix, qs.start, qs.bases)
    idx = list(range(0, qs.n, max(1, qs.n // n_sample)))[:n_sample]
    if qs.n - 1 not in idx:
        idx.append(qs.n - 1)  # the last query ends the batch (ragged tail)
    ox = oracle.Index(bank, k=11, stride=stride)
    ref = ox.search(qs.subset(idx), oracle.Params(stride=stride), threads=os.cpu_count() or 1)
    n_aln = 0
    for j, qi in enumerate(idx):
        got, exp = res.query(qi), ref[j].ranked
        assert len(got) == len(exp), f"query {qi}: {len(got)} vs {len(exp)} alignments"
        for fg, fe in FIELDS:
            assert np.array_equal(got[fg].astype(np.int64), exp[fe].astype(np.int64)), f"query {qi} field {fg}"
        tiny = (np.abs(got["evalue"]) < 1e-300) & (np.abs(exp["evalue"]) < 1e-300)
        assert (tiny | np.isclose(got["evalue"], exp["evalue"], rtol=1e-9, atol=0)).all(), f"query {qi} evalue"
        n_aln += len(got)
    ix.close()
    return n_aln


def test_mid_config_sampled(gn):
    bank = synth.make_bank("mid")
    qs = synth.make_queries("mid", bank)
    assert qs.n == 1000
    assert compare_sampled(gn, bank, qs, 60) > 500


def test_batched_config_sampled(gn):
    bank = synth.make_bank("batched")
    qs = synth.make_queries("batched", bank)
    assert qs.n == 10000
    assert compare_sampled(gn, bank, qs, 120) > 500


def test_large_config_sampled(gn):
    bank = synth.make_bank("large")
    qs = synth.make_queries("large", bank)
    assert qs.n == 2000
    assert compare_sampled(gn, bank, qs, 40) > 500
