"""Pins for the oracle's index build ("Inverted Indexes" section of the paper)."""
import itertools
import json
import os
import random

import numpy as np
import pytest

import oracle
import synth
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_seq(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


def _bank_with_oddities(rng, n=40):
    seqs = []
    for i in range(n):
        L = rng.randint(0, 60)
        s = list(_rand_seq(rng, L))
        if L and i % 5 == 0:                      # non-bases are never indexed
            s[rng.randrange(L)] = "N"
        if L and i % 7 == 0:                      # lower case and RNA letters are bases
            j = rng.randrange(L)
            s[j] = rng.choice("acgtu")
        seqs.append("".join(s))
    return seqs


@pytest.mark.parametrize("k,t", [(3, 3), (3, 1), (4, 2), (5, 5), (2, 7)])
def test_buckets_equal_bruteforce_listing(k, t):
    """Every bucket lists exactly the bank windows equal to the bucket's k-mer, in
    (seq, pos) order, and bucket i belongs to the i-th k-mer in A<C<G<T
    lexicographic order (itertools.product enumerates them independently of
    any 2-bit arithmetic)."""
    rng = random.Random(1000 + 10 * k + t)
    seqs = _bank_with_oddities(rng)
    bank = synth.bank_from_strings(seqs)
    ix = oracle.Index(bank, k=k, stride=t)
    bs, ps, pp = ix.buckets()
    brute = _brute.bank_windows(seqs, k, t)
    assert ix.n_postings == sum(len(v) for v in brute.values())
    for i, kmer in enumerate(itertools.product("ACGT", repeat=k)):
        w = "".join(kmer)
        got = list(zip(ps[bs[i]:bs[i + 1]].tolist(), pp[bs[i]:bs[i + 1]].tolist()))
        assert got == brute.get(w, []), (i, w)


@pytest.mark.parametrize("t", [1, 5, 11, 18])
def test_posting_count_equals_window_rule(t):
    """Posting count = sum over sequences of floor((len-k)/t)+1 (len >= k) on an all-ACGT bank."""
    bank = synth.make_bank("tiny")
    k = 11
    ix = oracle.Index(bank, k=k, stride=t)
    L = np.diff(bank.seq_start.astype(np.int64))
    expect = int(np.sum(np.where(L >= k, (L - k) // t + 1, 0)))
    assert ix.n_postings == expect


def test_paper_index_size_example():
    """Worked example of the index memory model: 4 Gbp at 11-base windows gives
    363 million windows and 2,833 MiB; 18-base (masked) windows give 222 million
    and 1,759 MiB.  Window count follows the same rule the oracle indexes by
    (pinned above), with 8 bytes per occurrence and 16 bytes per bucket."""
    g = json.load(open(os.path.join(GOLDEN, "index_size_example.json")))
    l, s = g["bank_bases"], g["sub_sequence_length"]
    for case in g["cases"]:
        m = case["window_length"]
        windows = (l - m) // m + 1                 # one long sequence, stride = window length
        assert round(windows / 1e6) in (case["windows_printed_millions"], case["windows_printed_millions"] + 1)
        mib_printed = case["windows_printed_millions"] * 1e6 * 8 / 2**20 + 4**s * 16 / 2**20
        mib_exact = windows * 8 / 2**20 + 4**s * 16 / 2**20
        # the paper's rounding of the window count moves the result by < 6 MiB
        assert abs(mib_printed - case["index_mib_printed"]) < 2.0 or abs(mib_exact - case["index_mib_printed"]) < 2.0
    # 8 bytes per occurrence in the oracle (two 4-byte integers, as the paper states)
    ix = oracle.Index(synth.bank_from_strings(["ACGTACGTACGTACGT"]), k=4, stride=4)
    _, ps, pp = ix.buckets()
    assert ps.itemsize + pp.itemsize == 8
    # bucket table: 4^11 entries of 8 bytes = 32 MiB ("Parallelization Methods")
    assert 4**11 * 8 / 2**20 == g["bucket_table_bytes_per_fragment_printed_mib"]


def test_short_and_empty_sequences():
    bank = synth.bank_from_strings(["", "ACG", "ACGTACGTACG", "NNNNNNNNNNNNNNNNNN"])
    ix = oracle.Index(bank, k=11, stride=11)
    assert ix.n_postings == 1
    bs, ps, pp = ix.buckets()
    assert ps.tolist() == [2] and pp.tolist() == [0]


def test_invalid_k_rejected():
    bank = synth.bank_from_strings(["ACGT"])
    with pytest.raises(ValueError):
        oracle.Index(bank, k=0, stride=1)
    with pytest.raises(ValueError):
        oracle.Index(bank, k=17, stride=1)


# ------------------------------------------------------------ spaced seeds --
@pytest.mark.parametrize("mask,t", [("1101", 4), ("1101", 1), ("10111", 3), ("110011", 6), ("1", 2)])
def test_masked_buckets_equal_bruteforce_listing(mask, t):
    """With a mask ("Methods": PatternHunter-style seeds) a window covers the mask's
    length and is indexed under its kept bases; bucket i is the i-th kept-base string
    in A<C<G<T order."""
    rng = random.Random(77 + len(mask) + t)
    seqs = _bank_with_oddities(rng)
    bank = synth.bank_from_strings(seqs)
    ix = oracle.Index(bank, stride=t, mask=mask)
    k = mask.count("1")
    assert ix.k == k
    bs, ps, pp = ix.buckets()
    brute = _brute.masked_windows(seqs, mask, t)
    assert ix.n_postings == sum(len(v) for v in brute.values())
    for i, kmer in enumerate(itertools.product("ACGT", repeat=k)):
        w = "".join(kmer)
        got = list(zip(ps[bs[i]:bs[i + 1]].tolist(), pp[bs[i]:bs[i + 1]].tolist()))
        assert got == brute.get(w, []), (mask, i, w)


def test_masked_paper_mask_window_rule():
    """The paper's mask 111010010100110111 keeps 11 of 18 bases; at stride 18 the
    posting count is sum(floor((len-18)/18)+1) on an all-ACGT bank, and a plain mask of
    k ones is the plain index."""
    bank = synth.make_bank("tiny")
    mask = "111010010100110111"
    ix = oracle.Index(bank, stride=18, mask=mask)
    assert ix.k == 11
    L = np.diff(bank.seq_start.astype(np.int64))
    assert ix.n_postings == int(np.sum(np.where(L >= 18, (L - 18) // 18 + 1, 0)))
    a = oracle.Index(bank, k=7, stride=5).buckets()
    b = oracle.Index(bank, stride=5, mask="1111111").buckets()
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_masked_rejects_bad_masks():
    bank = synth.bank_from_strings(["ACGTACGT"])
    for bad in ("", "0000", "1" * 17, "1" * 33, "1021"):
        with pytest.raises(ValueError):
            oracle.Index(bank, stride=1, mask=bad)


@pytest.mark.parametrize("stride,mask", [(11, None), (1, None), (6, "111010010100110111")])
def test_restricted_index_equals_full_on_kept_buckets(stride, mask):
    """The index restricted to some queries' seed codes holds, for every such code, the full
    index's bucket (same occurrences, same order) and nothing else; searching those queries
    gives the full index's results.  Several scan threads give the same index as one."""
    bank = synth.make_bank("mid", n_seqs=3000)
    qs = synth.make_queries("mid", bank, n=6)
    full = oracle.Index(bank, k=11, stride=stride, mask=mask)
    bs, ps, pp = full.buckets()
    keep = set()
    span = len(mask) if mask else 11
    for i in range(qs.n):
        q = qs.query(i)
        for x in range(len(q) - span + 1):
            w = q[x:x + span].decode()
            kept = _brute.kept(w, mask) if mask else "".join(_brute.norm(c) for c in w)
            if all(_brute.is_base(c) for c in kept):
                keep.add(kept)
    kept_codes = set()
    for s in keep:
        c = 0
        for ch in s:
            c = 4 * c + "ACGT".index(ch)
        kept_codes.add(c)
    for threads in (1, 5):
        r = oracle.Index(bank, k=11, stride=stride, mask=mask, restrict_to=qs, threads=threads)
        rbs, rps, rpp = r.buckets()
        counts = np.diff(rbs)
        assert set(np.nonzero(counts)[0].tolist()) <= kept_codes
        for c in kept_codes:
            a, b = int(bs[c]), int(bs[c + 1])
            ra, rb = int(rbs[c]), int(rbs[c + 1])
            assert np.array_equal(ps[a:b], rps[ra:rb]) and np.array_equal(pp[a:b], rpp[ra:rb]), c
        p = oracle.Params(stride=stride)
        got, exp = r.search(qs, p), full.search(qs, p)
        for g, e in zip(got, exp):
            assert np.array_equal(g.ranked, e.ranked)
