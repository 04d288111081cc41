"""The long-query reading, checked on the CPU with brute-force hits.

Queries longer than a segment are searched in overlapping segments and the chain
pieces are joined: a piece joins the chain on its (sequence, diagonal) when its first
hit starts no later than the chain's last hit (qs + k <= qe), and min_hsp_len applies
after the join.  Here the segment geometry is scaled down (segments of S bases that
overlap by V, D + k <= V) and the result is compared with the chains of the whole
query, which is the method's definition.  The repeat filter is included at its
strongest (a hit is dropped unless another hit of its diagonal lies within D offsets
inside its segment): the filters of the search only ever drop such hits."""
import random

import pytest

from tests import _brute


def _rand(rng, n):
    return "".join(rng.choice("ACGT") for _ in range(n))


def _mutate(rng, s, p_sub):
    return "".join(c if rng.random() >= p_sub else rng.choice("ACGT".replace(c, "")) for c in s)


def segmented_chains(seqs, query, k, t, D, min_len, S, V, filt):
    step = S - V
    pieces = []
    o = 0
    while True:
        seg = query[o:o + S]
        hl = _brute.hits(seqs, seg, k, t)
        if filt:
            diag = {}
            for qp, s, p in hl:
                diag.setdefault((s, p - qp), []).append(qp)
            hl = [(qp, s, p) for qp, s, p in hl if any(x != qp and abs(x - qp) <= D for x in diag[(s, p - qp)])]
        for s, a, b, ds, de, ln in _brute.chains(hl, k, D, 1):
            pieces.append((s, ds - (a + o), a + o, b + o))  # sequence, diagonal, qs, qe of the query
        if o + S >= len(query):
            break
        o += step
    pieces.sort()
    joined = []
    for s, d, a, b in pieces:
        if joined and joined[-1][0] == s and joined[-1][1] == d and a + k <= joined[-1][3]:
            joined[-1][3] = max(joined[-1][3], b)
        else:
            joined.append([s, d, a, b])
    return sorted((s, a, b, a + d, b + d, b - a) for s, d, a, b in joined if b - a >= min_len)


@pytest.mark.parametrize("D,min_len,filt", [(33, 22, True), (33, 22, False), (49, 44, True), (33, 11, False),
                                            (5, 11, False), (20, 33, True)])
def test_segments_joined_equal_whole_query_chains(D, min_len, filt):
    k, t, S, V = 11, 11, 300, 60
    assert D + k <= V
    rng = random.Random(1000 + D + min_len)
    seqs = [_rand(rng, rng.randint(150, 400)) for _ in range(25)]
    # a repeat family, so that several sequences share diagonals' worth of hits
    fam = _rand(rng, 120)
    for j in range(0, 25, 5):
        at = rng.randrange(0, len(seqs[j]) - 120)
        seqs[j] = seqs[j][:at] + _mutate(rng, fam, 0.05) + seqs[j][at + 120:]
    for trial in range(2):
        q = list(_rand(rng, 1300))
        # homologs across and beside the segment boundaries (segments start every S - V)
        for at in (S - V - 50, S - 30, 2 * (S - V) - 5, 2 * (S - V) + V - 40, 3 * (S - V) + 10, 700):
            src = seqs[rng.randrange(len(seqs))]
            a = rng.randrange(0, len(src) - 100)
            piece = _mutate(rng, src[a:a + rng.randint(60, 140)], 0.03)
            q[at:at + len(piece)] = piece
        q = "".join(q[:1300])
        whole = _brute.chains(_brute.hits(seqs, q, k, t), k, D, min_len)
        assert segmented_chains(seqs, q, k, t, D, min_len, S, V, filt) == whole
        assert whole, "the case plants homologs"


def test_join_needs_the_overlap():
    """With less overlap than D + k a chain can fall apart at a boundary: the bound is tight."""
    k, t, D, S = 11, 11, 33, 300
    rng = random.Random(7)
    seqs = [_rand(rng, 400)]
    src = seqs[0]
    q = _rand(rng, 258) + src[0:11] + _rand(rng, 22) + src[33:44] + _rand(rng, 400)  # hits at 258 and 291
    whole = _brute.chains(_brute.hits(seqs, q, k, t), k, D, 22)
    assert whole == [(0, 258, 302, 0, 44, 44)]
    # segments of 300 bases overlapping by 40 (< D + k): the first holds hit offsets up to
    # 289, the second starts at 260, so each hit lies in one segment only
    for filt in (True, False):
        assert segmented_chains(seqs, q, k, t, D, 22, S, 40, filt) == []
    # overlapping by 44 = D + k: the second segment starts at 256 and holds both hits
    assert segmented_chains(seqs, q, k, t, D, 22, S, 44, True) == whole
