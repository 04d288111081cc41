"""The seeded generator: deterministic, thread-count independent, shaped as its recipes state."""
import numpy as np

import synth


def test_deterministic_and_thread_independent():
    a = synth.make_bank("mid", n_seqs=3000, threads=1)
    b = synth.make_bank("mid", n_seqs=3000, threads=5)
    assert np.array_equal(a.seq_start, b.seq_start) and np.array_equal(a.bases, b.bases)
    qa = synth.make_queries("mid", a, n=50)
    qb = synth.make_queries("mid", b, n=50)
    assert np.array_equal(qa.bases, qb.bases) and np.array_equal(qa.start, qb.start)


def test_tiny_recipe():
    bank = synth.make_bank("tiny")
    L = np.diff(bank.seq_start.astype(np.int64))
    assert bank.n_seqs == 1000 and L.min() >= 500 and L.max() <= 2000
    assert set(np.unique(bank.bases).tolist()) <= set(b"ACGT")
    q = synth.make_queries("tiny", bank)
    ql = np.diff(q.start.astype(np.int64))
    assert q.n == 10 and ql.min() >= 250 and ql.max() <= 1100
    assert q.meta[:, 0].all()


def test_mid_recipe_shape():
    bank = synth.make_bank("mid", n_seqs=20000)
    L = np.diff(bank.seq_start.astype(np.int64))
    assert L.min() >= 100 and L.max() <= 50000
    assert 1350 < np.median(L) < 1650
    assert 1800 < L.mean() < 2200                 # ~400 Mbp at 200,000 sequences
    q = synth.make_queries("batched", bank, n=2000)
    ql = np.diff(q.start.astype(np.int64))
    assert ql.min() >= 40 and ql.max() <= 6000
    assert 0.45 < q.meta[:, 0].mean() < 0.55


def test_poisson_arrivals():
    t = synth.poisson_arrivals(200.0, 4000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all() and abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0


def test_long_query_recipe():
    """Random queries of the long recipe span 65,536 bp - 1 Mbp; planted homologs are clipped to the
    longest bank sequence (here the tiny bank's)."""
    bank = synth.make_bank("tiny")
    qs = synth.make_queries("long", bank)
    lens = np.diff(qs.start).astype(np.int64)
    planted = qs.meta[:, 0] != 0
    assert qs.n == 40 and 0 < planted.sum() < 40
    assert ((lens[~planted] >= 65_536) & (lens[~planted] <= 1_000_000)).all()
    longest = int(np.diff(bank.seq_start).max())
    assert (qs.meta[planted, 3] <= longest).all()
    again = synth.make_queries("long", bank)
    assert np.array_equal(again.bases, qs.bases)
