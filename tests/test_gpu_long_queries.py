"""Queries longer than 65,535 bases (the paper's query sets reach 1 Mbp).

The seed phases take such a query in overlapping segments and join the chain
pieces afterwards; the result must be exactly the method's result on the whole
query, which the oracle computes without any segmentation.  The cases plant
homologs across the segment boundaries (every 57,343 bases), an exact copy longer
than 65,535 bases (one HSP and one alignment longer than a segment), and mix
long and short queries in one call."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
          ("score", "score"), ("rank", "rank"))
SEG_STEP = 65535 - 8192


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


def _rand(rng, n):
    return bytes(rng.choice(np.frombuffer(b"ACGT", dtype=np.uint8), n))


def _mutate(rng, s, p_sub, p_indel):
    out = bytearray()
    for c in s:
        u = rng.random()
        if u < p_indel / 2:
            continue  # deletion
        if u < p_indel:
            out += _rand(rng, 1)  # insertion before the base
        out.append(c if rng.random() >= p_sub else b"ACGT"[(b"ACGT".index(c) + rng.integers(1, 4)) % 4])
    return bytes(out)


def make_long_case():
    rng = np.random.default_rng(0x10A6)
    seqs = [_rand(rng, int(rng.integers(800, 3000))) for _ in range(300)]
    seqs.append(_rand(rng, 180_000))  # sequence 300: source of the long homologs
    seqs.append(_rand(rng, 70_000))
    bank = synth.bank_from_strings(seqs)
    big = seqs[300]
    # q0: a 100 kbp diverged copy crossing two segment boundaries, in random flanks
    q0 = _rand(rng, 20_000) + _mutate(rng, big[10_000:110_000], 0.03, 0.005) + _rand(rng, 30_000)
    # q1: short homologs planted across and near the boundaries of a 200 kbp random query
    q1 = bytearray(_rand(rng, 200_000))
    for at in (SEG_STEP - 400, SEG_STEP + 8192 - 250, 2 * SEG_STEP - 1000, 2 * SEG_STEP + 8000, 3 * SEG_STEP - 60,
               65535 - 40, 100_000):
        src = seqs[int(rng.integers(0, 300))]
        piece = _mutate(rng, src[:min(len(src), 900)], 0.04, 0.01)
        q1[at:at + len(piece)] = piece
    q1 = bytes(q1[:200_000])
    # q2: an ordinary short query; q3: an exact copy longer than one segment
    q2 = _mutate(rng, seqs[7], 0.05, 0.01)
    q3 = big[30_000:100_000]
    # q4: 65,536 bases, one more than a segment holds
    q4 = _rand(rng, 60_000) + big[150_000:155_536]
    qs = synth.queries_from_strings([q0, q1, q2, q3, q4])
    return bank, qs


@pytest.fixture(scope="module")
def long_case():
    return make_long_case()


def _compare(gn, res, ref, n, what):
    n_aln = 0
    for i in range(n):
        got, exp = res.query(i), ref[i].ranked
        assert len(got) == len(exp), f"{what} query {i}: {len(got)} vs {len(exp)} alignments"
        for fg, fe in FIELDS:
            assert np.array_equal(got[fg].astype(np.int64), exp[fe].astype(np.int64)), f"{what} query {i} field {fg}"
        tiny = (np.abs(got["evalue"]) < 1e-300) & (np.abs(exp["evalue"]) < 1e-300)
        assert (tiny | np.isclose(got["evalue"], exp["evalue"], rtol=1e-9, atol=0)).all(), f"{what} query {i}"
        n_aln += len(got)
    return n_aln


@pytest.mark.parametrize("kw", [dict(), dict(min_hsp_len=11), dict(min_hsp_len=44), dict(max_hit_distance=100),
                                dict(max_alignments=0), dict(band_w=40)])
def test_long_queries_equal_oracle(gn, long_case, kw):
    bank, qs = long_case
    ix = gn.Index.from_bank(bank)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(**kw))
    ref = oracle.Index(bank).search(qs, oracle.Params(**kw), threads=os.cpu_count() or 1)
    assert _compare(gn, res, ref, qs.n, kw) > 5
    # the exact copy: one alignment over the whole query, longer than a segment
    top = res.query(3)[0]
    assert top["seq"] == 300 and top["q_start"] == 0 and top["q_end"] == 70_000 and top["score"] == 70_000
    ix.close()


def test_long_queries_masked_and_both_strands(gn, long_case):
    bank, qs = long_case
    mask = "111010010100110111"
    ix = gn.Index.from_bank(bank, stride=18, mask=mask)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_BOTH_STRANDS))
    ox = oracle.Index(bank, k=11, stride=18, mask=mask)
    ref = ox.search(qs, oracle.Params(stride=18, both_strands=True), threads=os.cpu_count() or 1)
    assert res.n_queries == 2 * qs.n
    assert _compare(gn, res, ref, 2 * qs.n, "masked both strands") > 5
    ix.close()


def test_long_query_equals_its_segments_alone_when_short(gn, long_case):
    """A batch of short queries gives the same results with and without a long query in it."""
    bank, qs = long_case
    ix = gn.Index.from_bank(bank)
    short = qs.subset([2])
    a = gn.search(ix, short.start, short.bases).query(0)
    b = gn.search(ix, qs.start, qs.bases).query(2)
    assert len(a) == len(b) and all(np.array_equal(a[f], b[f]) for f, _ in FIELDS)
    ix.close()


def test_long_query_limits(gn, long_case):
    bank, qs = long_case
    ix = gn.Index.from_bank(bank)
    q = qs.subset([0])
    with pytest.raises(gn.GnError) as e:  # the seed distance must fit the segments' overlap
        gn.search(ix, q.start, q.bases, params=gn.make_params(max_hit_distance=9000))
    assert e.value.status == gn.GN_EINVAL
    with pytest.raises(gn.GnError) as e:
        gn.search(ix, q.start, q.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    assert e.value.status == gn.GN_EINVAL
    big = synth.queries_from_strings([b"A" * (1 << 24)])
    with pytest.raises(gn.GnError) as e:
        gn.search(ix, big.start, big.bases)
    assert e.value.status == gn.GN_ETOOBIG
    ix.close()
