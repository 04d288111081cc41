"""Pins for the oracle's search phases ("Searching process" section of the paper)."""
import random

import numpy as np
import pytest

import oracle
import synth
from tests import _brute

P = oracle.Params()


def _rand(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


def _mutate(rng, s, p_sub, p_indel):
    out = []
    for c in s:
        u = rng.random()
        if u < p_indel:
            if rng.random() < 0.5:
                out.append(rng.choice("ACGT"))
                out.append(c)
        elif u < p_indel + p_sub:
            out.append(rng.choice([b for b in "ACGT" if b != c]))
        else:
            out.append(c)
    return "".join(out)


# ------------------------------------------------------------ phases 1-2 --
@pytest.mark.parametrize("k,t", [(4, 4), (5, 1), (6, 3)])
def test_hits_equal_bruteforce(k, t):
    """Every (query offset, bank window) pair with equal k-base strings is a hit, and nothing else."""
    rng = random.Random(7 + k * t)
    seqs = [_rand(rng, rng.randint(0, 80)) for _ in range(30)]
    seqs[3] = seqs[3][:10] + "N" + seqs[3][11:]
    bank = synth.bank_from_strings(seqs)
    ix = oracle.Index(bank, k=k, stride=t)
    for trial in range(4):
        q = _rand(rng, rng.randint(0, 60))
        if trial == 1 and len(q) > 5:
            q = q[:5] + "N" + q[6:]
        r = ix.search_one(q.encode(), oracle.Params(k=k, stride=t, keep_hits=True))
        brute = sorted(_brute.hits(seqs, q, k, t))
        got = sorted((int(h["qpos"]), int(h["seq"]), int(h["pos"])) for h in r.hits)
        assert got == brute
        assert r.n_hits == len(brute)
        # the exported list is in (seq, diagonal, qpos) order
        keys = [(int(h["seq"]), int(h["pos"]) - int(h["qpos"]), int(h["qpos"])) for h in r.hits]
        assert keys == sorted(keys)


@pytest.mark.parametrize("k,t,D,min_len", [(4, 4, 12, 8), (5, 1, 3, 5), (4, 2, 6, 10), (6, 3, 9, 6)])
def test_hsps_equal_bruteforce_chains(k, t, D, min_len):
    """HSPs = maximal runs of hits on one (sequence, diagonal) with query gaps <= D, length >= min."""
    rng = random.Random(99 + k + D)
    seqs = [_rand(rng, rng.randint(20, 200)) for _ in range(20)]
    bank = synth.bank_from_strings(seqs)
    ix = oracle.Index(bank, k=k, stride=t)
    for trial in range(5):
        s = seqs[rng.randrange(len(seqs))]
        a = rng.randrange(0, len(s) - 10)
        q = _mutate(rng, s[a:a + rng.randint(10, 120)], 0.08, 0.02) + _rand(rng, 10)
        params = oracle.Params(k=k, stride=t, max_hit_distance=D, min_hsp_len=min_len, keep_hits=True)
        r = ix.search_one(q.encode(), params)
        expect = _brute.chains(_brute.hits(seqs, q, k, t), k, D, min_len)
        got = sorted(tuple(int(x) for x in h) for h in r.hsp)
        assert got == expect


def test_hsp_hand_case_exact_copy():
    """Query = bank[22:122] of a 200-base sequence, k = t = 11: windows at 22, 33, ..., 110 lie
    inside the copy, so 9 hits on diagonal 22 form the HSP q[0, 99) x db[22, 121), length 99."""
    rng = random.Random(5)
    s = _rand(rng, 200)
    bank = synth.bank_from_strings([s])
    ix = oracle.Index(bank, k=11, stride=11)
    r = ix.search_one(s[22:122].encode(), oracle.Params(keep_hits=True))
    on_diag = [h for h in r.hits if int(h["pos"]) - int(h["qpos"]) == 22]
    assert [int(h["qpos"]) for h in on_diag] == list(range(0, 89, 11))
    assert (0, 0, 99, 22, 121, 99) in [tuple(int(x) for x in h) for h in r.hsp]


def test_hsp_hand_case_distance_parameter():
    """Hits at query offsets 0, 11, 44, 55 (windows 22 and 33 broken by one substitution each):
    the 33-base gap joins them when D = 33 and splits them when D = 32."""
    rng = random.Random(6)
    s = _rand(rng, 66)
    q = list(s)
    for pos in (27, 38):                       # one change inside window 22..32 and 33..43
        q[pos] = "A" if q[pos] != "A" else "C"
    q = "".join(q)
    bank = synth.bank_from_strings([s])
    ix = oracle.Index(bank, k=11, stride=11)
    r = ix.search_one(q.encode(), oracle.Params(max_hit_distance=33, min_hsp_len=22, keep_hits=True))
    assert [tuple(int(x) for x in h) for h in r.hsp] == [(0, 0, 66, 0, 66, 66)]
    r = ix.search_one(q.encode(), oracle.Params(max_hit_distance=32, min_hsp_len=22, keep_hits=True))
    assert sorted(tuple(int(x) for x in h) for h in r.hsp) == [(0, 0, 22, 0, 22, 22), (0, 44, 66, 44, 66, 22)]


# ---------------------------------------------------------------- phase 3 --
def _ext_case(left_flank_q, left_flank_s, core, right_flank_q, right_flank_s, params=P):
    q = left_flank_q + core + right_flank_q
    s = left_flank_s + core + right_flank_s
    hsp = (len(left_flank_q), len(left_flank_q) + len(core), len(left_flank_s), len(left_flank_s) + len(core))
    return oracle.extend(q, s, hsp, params)


def test_extension_stops_after_xdrop():
    """10 matches then 7 mismatches (score 10 -> -11, drop 21 > 20): the end moves by 10."""
    core = "ACGTACGTACGTACGTACGTAC"
    rq = "GATTACAGAT" + "AAAAAAA" + "CCCCCCCCCCCC"
    rs = "GATTACAGAT" + "TTTTTTT" + "CCCCCCCCCCCC"
    assert _ext_case("", "", core, rq, rs) == (0, 32, 0, 32)


def test_extension_crosses_shallow_dip():
    """10 matches, 6 mismatches (drop 18 <= 20), 30 matches: the end moves by 46."""
    core = "ACGTACGTACGTACGTACGTAC"
    m30 = "GCTAGCTAGCTAGCTAGCTAGCTAGCTAGC"
    rq = "GATTACAGAT" + "AAAAAA" + m30 + "A" * 10
    rs = "GATTACAGAT" + "TTTTTT" + m30 + "T" * 10
    assert _ext_case("", "", core, rq, rs) == (0, 22 + 46, 0, 22 + 46)


def test_extension_drop_equal_to_x_continues():
    """With mismatch -4, 5 mismatches drop exactly X = 20 (not more): the walk goes on; 6 stop it."""
    p = oracle.Params(mismatch=-4)
    core = "ACGTACGTACGTACGTACGTAC"
    m30 = "GCTAGCTAGCTAGCTAGCTAGCTAGCTAGC"
    rq = "GATTACAGAT" + "AAAAA" + m30
    rs = "GATTACAGAT" + "TTTTT" + m30
    assert _ext_case("", "", core, rq, rs, p) == (0, 22 + 45, 0, 22 + 45)
    rq = "GATTACAGAT" + "AAAAAA" + m30
    rs = "GATTACAGAT" + "TTTTTT" + m30
    assert _ext_case("", "", core, rq, rs, p) == (0, 32, 0, 32)
    # the same on the left end (flanks read right to left from the core)
    lq = m30 + "AAAAA" + "GATTACAGAT"
    ls = m30 + "TTTTT" + "GATTACAGAT"
    assert _ext_case(lq, ls, core, "", "", p) == (0, 45 + 22, 0, 45 + 22)
    lq = m30 + "AAAAAA" + "GATTACAGAT"
    ls = m30 + "TTTTTT" + "GATTACAGAT"
    assert _ext_case(lq, ls, core, "", "", p) == (36, 36 + 32, 36, 36 + 32)


def test_extension_first_best_and_left_side():
    """Left: 5 matches, 1 mismatch, 3 matches then mismatches: scores 5, 2, 5 -> the first best (5)
    is kept.  The walk also stops at the start of either sequence."""
    core = "ACGTACGTACGTACGTACGTAC"
    # left flanks read right-to-left from the core: 5 matches, mismatch, 3 matches, 8 mismatches
    lq = "AAAAAAAA" + "GCA" + "G" + "TTACG"
    ls = "CCCCCCCC" + "GCA" + "C" + "TTACG"
    assert _ext_case(lq, ls, core, "", "") == (len(lq) - 5, len(lq) + 22, len(ls) - 5, len(ls) + 22)
    # all matches up to the query start: extends to 0
    assert _ext_case("GATTACA", "TTGATTACA", core, "", "") == (0, 29, 2, 31)


def test_extension_non_bases_are_mismatches():
    core = "ACGTACGTACGTACGTACGTAC"
    # N against N is not a match: 'NNNNNNN' = 7 mismatches -> drop 21 > 20 before the matches
    rq = "NNNNNNN" + "ACGTACGTAC"
    rs = "NNNNNNN" + "ACGTACGTAC"
    assert _ext_case("", "", core, rq, rs) == (0, 22, 0, 22)


# ---------------------------------------------------------------- phase 4 --
def test_overlap_merge_hand_cases():
    m = oracle.merge_overlaps
    # both ranges intersect -> union box
    assert m([(0, 0, 10, 0, 10), (0, 5, 15, 5, 15)]) == [(0, 0, 15, 0, 15)]
    # query ranges intersect, bank ranges do not -> two boxes
    assert m([(0, 0, 10, 0, 10), (0, 5, 15, 50, 60)]) == [(0, 0, 10, 0, 10), (0, 5, 15, 50, 60)]
    # half-open ranges that only touch do not intersect
    assert m([(0, 0, 10, 0, 10), (0, 10, 20, 10, 20)]) == [(0, 0, 10, 0, 10), (0, 10, 20, 10, 20)]
    # query ranges only touch while bank ranges overlap -> still two boxes (both must intersect)
    assert m([(0, 0, 10, 0, 10), (0, 10, 20, 5, 15)]) == [(0, 0, 10, 0, 10), (0, 10, 20, 5, 15)]
    # bank ranges only touch while query ranges overlap -> two boxes
    assert m([(0, 0, 10, 0, 10), (0, 5, 15, 10, 20)]) == [(0, 0, 10, 0, 10), (0, 5, 15, 10, 20)]
    # different bank sequences never merge
    assert m([(1, 0, 10, 0, 10), (0, 0, 10, 0, 10)]) == [(0, 0, 10, 0, 10), (1, 0, 10, 0, 10)]
    # a third HSP that meets only the union of the first two still joins it
    assert m([(0, 0, 10, 0, 10), (0, 8, 30, 8, 30), (0, 25, 40, 28, 44)]) == [(0, 0, 40, 0, 44)]
    # single sweep: C meets the closed box A, but is compared with the current box B only
    assert m([(0, 0, 10, 0, 10), (0, 5, 15, 100, 110), (0, 8, 20, 5, 12)]) == \
        [(0, 0, 10, 0, 10), (0, 5, 15, 100, 110), (0, 8, 20, 5, 12)]
    # input order does not matter (the sweep sorts by qs, ds, qe, de)
    assert m([(0, 8, 30, 8, 30), (0, 25, 40, 28, 44), (0, 0, 10, 0, 10)]) == [(0, 0, 40, 0, 44)]


def test_overlap_merge_invariants():
    rng = random.Random(3)
    for _ in range(50):
        hs = []
        for _ in range(rng.randint(1, 12)):
            qs = rng.randint(0, 80); ds = rng.randint(0, 80)
            ln = rng.randint(1, 25)
            hs.append((rng.randint(0, 2), qs, qs + ln, ds, ds + ln + rng.randint(-3, 3) if ln > 3 else ds + ln))
        out = oracle.merge_overlaps(hs)
        # every input lies inside exactly one output box of its sequence that was built from it
        for (s, qs, qe, ds, de) in hs:
            assert any(o[0] == s and o[1] <= qs and qe <= o[2] and o[3] <= ds and de <= o[4] for o in out)
        assert len(out) <= len(hs)
        # consecutive boxes of one sequence in sweep order do not intersect in both ranges
        for a, b in zip(out, out[1:]):
            if a[0] == b[0]:
                assert not (b[1] < a[2] and a[1] < b[2] and b[3] < a[4] and a[3] < b[4])


# ---------------------------------------------------------------- phase 6 --
def _full_box(q, s):
    return (0, len(q), 0, len(s))


def test_sw_equals_enumerated_local_alignment():
    """With a band wider than both sequences, banded SW = the best local alignment over all
    substring pairs and all alignments (exhaustive enumeration, strings up to 4 bases)."""
    rng = random.Random(11)
    wide = oracle.Params(band_w=64)
    for _ in range(60):
        a = _rand(rng, rng.randint(1, 4)); b = _rand(rng, rng.randint(1, 4))
        got = oracle.banded_sw(a, b, _full_box(a, b), wide)[0]
        assert got == _brute.local_score_enumerated(a, b), (a, b)


def test_sw_equals_suffix_recursion_on_longer_strings():
    """Strings up to 14 bases (with gaps worth taking): best local score = max over substring
    pairs of the best global score from an independent suffix recursion."""
    rng = random.Random(12)
    wide = oracle.Params(band_w=64)
    for _ in range(25):
        base = _rand(rng, rng.randint(6, 14))
        a = base; b = _mutate(rng, base, 0.1, 0.15)
        if not b:
            continue
        best = 0
        for i0 in range(len(a)):
            for i1 in range(i0 + 1, len(a) + 1):
                for j0 in range(len(b)):
                    for j1 in range(j0 + 1, len(b) + 1):
                        best = max(best, _brute.global_score(a[i0:i1], b[j0:j1]))
        assert oracle.banded_sw(a, b, _full_box(a, b), wide)[0] == best, (a, b)


def test_sw_hand_cases():
    rng = random.Random(13)
    wide = oracle.Params(band_w=300)
    s = _rand(rng, 200)
    # identical strings: score = length, whole ranges
    assert oracle.banded_sw(s, s, (0, 200, 0, 200), P) == (200, 0, 200, 0, 200)
    # one mismatch in the middle of 31 bases: 15 - 3 + 15 = 27
    a = "ACGTACGTACGTACG" + "A" + "TTGCATTGCATTGCA"
    b = "ACGTACGTACGTACG" + "C" + "TTGCATTGCATTGCA"
    assert oracle.banded_sw(a, b, (0, 31, 0, 31), P) == (27, 0, 31, 0, 31)
    # 200-base copy with one base deleted in the middle: 199 matches and a gap of 1: 199 - 7 = 192
    t = s[:100] + s[101:]
    assert oracle.banded_sw(s, t, (0, 200, 0, 199), wide)[0] == 192
    assert oracle.banded_sw(t, s, (0, 199, 0, 200), wide)[0] == 192
    # a 3-base deletion in either sequence: 197 matches and one gap of 3: 197 - (5 + 3*2) = 186
    t3 = s[:100] + s[103:]
    assert oracle.banded_sw(s, t3, (0, 200, 0, 197), wide)[0] == 186
    assert oracle.banded_sw(t3, s, (0, 197, 0, 200), wide)[0] == 186
    # the DP window reaches w rows and columns beyond the HSP: an HSP given as [50, 150) on an
    # identical pair yields the alignment [34, 166) with w = 16
    assert oracle.banded_sw(s, s, (50, 150, 50, 150), P) == (132, 34, 166, 34, 166)
    # equal-score alignments: the one ending at the smallest query end, then smallest bank end
    assert oracle.banded_sw("ACG", "ACGTTTTTACG", (0, 3, 0, 11), wide) == (3, 0, 3, 0, 3)


def test_sw_start_tie_rules_hand_cases():
    """Where two alignments of equal score meet in one cell, the reading's tie order decides
    which start is reported: H takes the diagonal over E over F, and E and F take a gap opened
    from H over one extended.  Each pair below has two best alignments with different starts
    that merge at a single tie of one kind; the expected start is the one the rule picks.
    Cells are (query row i, bank column j), 0-based; scores +1/-3, a gap of g costs 5 + 2g."""
    wide = oracle.Params(band_w=64)

    # Diagonal over E.  b is a with one of the two Cs at a[7:9] deleted.  Alignment 1 starts at
    # (0,0): a[0:8] = b[0:8] (8), a[8] against a gap (-7), a[9:17] = b[8:16] (8): 9.
    # Alignment 2 starts at (8,7): a[8:17] = b[7:16] (9 matches): 9.  At cell (8,7) the fresh
    # diagonal step C/C (0 + 1) ties with E = H(7,7) - 7 = 8 - 7 = 1; the diagonal wins.
    a, b = "ATAGTTACCGATCAATT", "ATAGTTACGATCAATT"
    assert oracle.banded_sw(a, b, _full_box(a, b), wide) == (9, 8, 17, 7, 16)

    # E over F.  a = (CA)^5 + s, b = (AC)^5 + s with s = ACTCGCACC.  On diagonal +1,
    # a[0:9] = b[1:10] (9 matches from (0,1)); on diagonal -1, a[1:10] = b[0:9] (9 matches
    # from (1,0)).  At cell (9,9) the vertical gap after the first, E = 9 - 7 = 2, ties with
    # the horizontal gap after the second, F = 9 - 7 = 2, and the diagonal step is below them
    # (H(8,8) = 1, A/C: -2).  Both continue over s on diagonal 0: 2 + 9 = 11.  E wins: (0,1).
    a, b = "CACACACACAACTCGCACC", "ACACACACACACTCGCACC"
    assert oracle.banded_sw(a, b, _full_box(a, b), wide) == (11, 0, 19, 1, 19)

    # E: open over extend.  a = (AC)^6 + CCA + s, b = (AC)^6 + s, s = GATGTTAGATAA (12).
    # Alignment 1 from (0,0): (AC)^6 on both (12), a[12:15] against a gap of 3 (-11), s (12): 13.
    # Alignment 2 from (2,0): a[2:12] = b[0:10] (10), C/A (-3), C/C (+1), so H(13,11) = 8; a[14]
    # against a gap of 1 (-7); s (12): 13.  At cell (14,11) E can extend alignment 1's gap a
    # third time (E(13,11) - 2 = 3 - 2 = 1) or open from H(13,11) (8 - 7 = 1); the open wins.
    a, b = "ACACACACACACCCAGATGTTAGATAA", "ACACACACACACGATGTTAGATAA"
    assert oracle.banded_sw(a, b, _full_box(a, b), wide) == (13, 2, 27, 0, 24)

    # F: open over extend, the mirror image (query and bank swapped, so the gaps are horizontal):
    # at cell (11,14) F can extend the three-base gap (1) or open from H(11,13) = 8 (1).
    assert oracle.banded_sw(b, a, _full_box(b, a), wide) == (13, 0, 24, 2, 27)


def test_sw_band_zero_is_best_ungapped_segment():
    """w = 0 on an HSP of diagonal 0 leaves only the main diagonal: the score is the best
    ungapped segment (Kadane's maximum subarray over match/mismatch scores)."""
    rng = random.Random(14)
    for _ in range(30):
        a = _rand(rng, 60)
        b = _mutate(rng, a, 0.15, 0.05)[:60]
        n = min(len(a), len(b))
        got = oracle.banded_sw(a, b, (0, n, 0, n), oracle.Params(band_w=0))[0]
        assert got == _brute.kadane([_brute.pair(a[i], b[i], 1, -3) for i in range(n)])


def test_sw_score_recomputes_over_reported_ranges():
    """The reported score equals the best end-to-end alignment of the reported ranges inside the
    same band (independent recursion), for homologous pairs with indels."""
    rng = random.Random(15)
    for trial in range(12):
        a = _rand(rng, rng.randint(40, 120))
        b = _rand(rng, 15) + _mutate(rng, a, 0.08, 0.04) + _rand(rng, 10)
        hsp = (0, len(a), 15, 15 + len(a))
        w = 8
        score, qs, qe, ds, de = oracle.banded_sw(a, b, hsp, oracle.Params(band_w=w))
        assert score > 0
        d_s, d_e = hsp[2] - hsp[0], hsp[3] - hsp[1]
        band = (min(d_s, d_e) - w, max(d_s, d_e) + w)
        g = _brute.global_score(a[qs:qe], b[ds:de], diag_range=band, offset=(qs, ds))
        assert g == score, (trial, score, g)
        # and no higher-scoring alignment exists in the DP region: widening nothing can beat it
        assert oracle.banded_sw(a, b, hsp, oracle.Params(band_w=200))[0] >= score


# ---------------------------------------------------------------- phase 7 --
def test_lambda_closed_form():
    """For +1/-3 on uniform bases, lambda solves 1/4 e^l + 3/4 e^-3l = 1, i.e. x = e^-l is the root
    in (0, 1) of 3x^3 + 3x^2 + 3x - 1 = 0."""
    import math
    lam = oracle.ungapped_lambda(1, -3)
    x = math.exp(-lam)
    assert abs(3 * x**3 + 3 * x**2 + 3 * x - 1) < 1e-12
    assert abs(lam - P.lam) < 1e-6
    assert abs(0.25 * math.exp(lam) + 0.75 * math.exp(-3 * lam) - 1) < 1e-12


def test_evalue_and_bits_identities():
    """E = m n 2^-bits (bit score definition), E(0) = K m n, E(S+1)/E(S) = e^-lambda."""
    import math
    for S in (1, 10, 57, 200, 500):
        for m, n in ((300, 1.25e6), (5000, 4.0e9)):
            e = oracle.evalue(S, m, n, P)
            b = oracle.bits(S, P)
            assert math.isclose(e, m * n * 2.0 ** (-b), rel_tol=1e-12)
            assert math.isclose(oracle.evalue(S + 1, m, n, P) / e, math.exp(-P.lam), rel_tol=1e-12)
    assert math.isclose(oracle.evalue(0, 100, 1000, P), P.K * 100 * 1000, rel_tol=1e-15)
    assert oracle.bits(0, P) == pytest.approx(-math.log2(P.K))


def test_rank_order_and_duplicates():
    """Score descending, ties by (seq, q_start, db_start, q_end, db_end); a record with the same
    sequence and ranges as an earlier (better) one is dropped even when others sort between them;
    non-positive scores are dropped; the e-value cut applies after de-duplication."""
    alns = [(2, 0, 10, 0, 10, 5), (1, 0, 10, 0, 10, 9), (1, 0, 10, 0, 10, 5), (1, 0, 10, 0, 11, 5),
            (0, 3, 9, 3, 9, 7), (0, 2, 9, 3, 9, 7), (3, 0, 5, 0, 5, 0), (1, 0, 10, 0, 10, 9)]
    got = oracle.rank(alns, 100, 1000, P)
    assert got == [(1, 0, 10, 0, 10, 9, 0), (0, 2, 9, 3, 9, 7, 1), (0, 3, 9, 3, 9, 7, 2),
                   (1, 0, 10, 0, 11, 5, 3), (2, 0, 10, 0, 10, 5, 4)]
    cut = oracle.evalue(7, 100, 1000, P)
    got = oracle.rank(alns, 100, 1000, oracle.Params(max_evalue=cut))
    assert [g[5] for g in got] == [9, 7, 7]


# ------------------------------------------------------------ end to end --
@pytest.fixture(scope="module")
def tiny():
    bank = synth.make_bank("tiny")
    qs = synth.make_queries("tiny", bank)
    ix = oracle.Index(bank)
    return bank, qs, ix


def test_planted_homologs_recovered(tiny):
    bank, qs, ix = tiny
    res = ix.search(qs, P)
    found = 0
    for i, r in enumerate(res):
        src_seq, src_pos, src_len = (int(x) for x in qs.meta[i][1:4])
        if len(r.ranked) and int(r.ranked[0]["seq"]) == src_seq:
            top = r.ranked[0]
            if int(top["ds"]) < src_pos + src_len and src_pos < int(top["de"]):
                found += 1
    assert found >= 9


def test_ranked_invariants(tiny):
    bank, qs, ix = tiny
    res = ix.search(qs, P)
    n_bank = bank.n_bases
    for i, r in enumerate(res):
        q = qs.query(i).decode()
        m = len(q)
        keys = [(-int(a["score"]), int(a["seq"]), int(a["qs"]), int(a["ds"]), int(a["qe"]), int(a["de"]))
                for a in r.ranked]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
        assert [int(a["rank"]) for a in r.ranked] == list(range(len(r.ranked)))
        assert len(r.sel) <= P.max_alignments
        sel_keys = [(-int(h["len"]), int(h["seq"]), int(h["qs"]), int(h["ds"])) for h in r.sel]
        assert sel_keys == sorted(sel_keys)
        for a in r.ranked[:3]:
            assert a["evalue"] == pytest.approx(oracle.evalue(int(a["score"]), m, n_bank, P), rel=1e-12)
            s = bank.seq(int(a["seq"])).decode()
            # the score recomputes over the reported ranges (band wide enough to hold the path)
            g = _brute.global_score(q[a["qs"]:a["qe"]], s[a["ds"]:a["de"]]) if a["qe"] - a["qs"] < 130 else None
            if g is not None:
                assert g >= int(a["score"])


def test_threads_and_repeat_are_deterministic(tiny):
    bank, qs, ix = tiny
    r1 = ix.search(qs, P, threads=1)
    r4 = ix.search(qs, P, threads=4)
    for a, b in zip(r1, r4):
        assert np.array_equal(a.ranked, b.ranked) and np.array_equal(a.sel, b.sel)


def test_max_alignments_and_empty_query(tiny):
    bank, qs, ix = tiny
    r = ix.search_one(qs.query(0), oracle.Params(max_alignments=1))
    assert len(r.sel) == 1 and len(r.ranked) == 1
    r = ix.search_one(b"", P)
    assert r.n_hits == 0 and len(r.ranked) == 0
    r = ix.search_one(b"ACGTACG", P)           # shorter than k
    assert r.n_hits == 0


# ---------------------------------------------------------- both strands --
def test_reverse_complement_definition():
    rc = oracle.reverse_complement
    assert rc(b"") == b""
    assert rc(b"A") == b"T" and rc(b"C") == b"G" and rc(b"G") == b"C" and rc(b"T") == b"A"
    assert rc(b"U") == b"A" and rc(b"u") == b"a" and rc(b"acgt") == b"acgt"
    assert rc(b"AACGN") == b"NCGTT"          # reversed, complemented, non-base kept
    assert rc(b"ACGT") == b"ACGT"            # a reverse palindrome
    assert rc(b"GATTACA") == b"TGTAATC"
    import random
    r = random.Random(7)
    for _ in range(50):
        s = bytes(r.choice(b"ACGTNacgt") for _ in range(r.randint(0, 40)))
        assert rc(rc(s)) == s
        assert len(rc(s)) == len(s)


def test_both_strands_finds_reverse_complement_homolog():
    bank = synth.make_bank("tiny", n_seqs=300)
    src = bank.seq(42)[100:500]
    q_fwd, q_rev = src, oracle.reverse_complement(src)
    ox = oracle.Index(bank)
    res = ox.search([q_fwd, q_rev], oracle.Params(both_strands=True))
    assert len(res) == 4
    # forward copy: found on its own strand (result 0); its reverse complement on result 3
    for j in (0, 3):
        top = res[j].ranked[0]
        assert int(top["seq"]) == 42 and int(top["score"]) == 400, j
    # the reverse-complemented query is not found as given (result 2), and result 1 is the same
    # search as result 2's complement pair
    assert all(int(a["seq"]) != 42 or int(a["score"]) < 100 for a in res[2].ranked)
    assert [tuple(a) for a in res[1].ranked] == [tuple(a) for a in ox.search([q_rev], oracle.Params())[0].ranked]
    # plain search is the even half of the both-strand search
    plain = ox.search([q_fwd, q_rev], oracle.Params())
    assert [tuple(a) for a in plain[1].ranked] == [tuple(a) for a in res[2].ranked]


# ------------------------------------------------------------ spaced seeds --
@pytest.mark.parametrize("mask,t", [("1101101", 7), ("1101101", 1), ("110101", 6)])
def test_masked_hits_and_hsps_equal_bruteforce(mask, t):
    """Masked seeds: hits are the query windows at every offset that agree with a bank
    window at the kept positions; an HSP runs from its first seed to the end of its last
    (len(mask) bases)."""
    rng = random.Random(5 + t)
    bank = synth.make_bank("tiny", n_seqs=40 if t > 1 else 10)
    seqs = [bank.seq(i).decode() for i in range(bank.n_seqs)]
    src = seqs[3][50:350]
    q = "".join(c if rng.random() > 0.08 else rng.choice("ACGT") for c in src)
    ox = oracle.Index(bank, stride=t, mask=mask)
    p = oracle.Params(stride=t, keep_hits=True)
    r = ox.search([q.encode()], p)[0]
    got = sorted((int(h["qpos"]), int(h["seq"]), int(h["pos"])) for h in r.hits)
    assert got == sorted(_brute.masked_hits(seqs, q, mask, t))
    pr = p.resolved()
    span = len(mask)
    brute_hsp = _brute.chains(got, span, pr.max_hit_distance, pr.min_hsp_len)
    assert sorted(tuple(int(x[f]) for f in ("seq", "qs", "qe", "ds", "de", "len")) for x in r.hsp) == brute_hsp
    assert len(r.ranked) >= 1 and int(r.ranked[0]["seq"]) == 3


def test_spaced_seed_survives_mismatches_at_removed_positions():
    """The point of the mask: a window with mismatches only where the mask removes bases
    still hits."""
    mask = "111010010100110111"
    rng = random.Random(9)
    w = "".join(rng.choice("ACGT") for _ in range(18))
    v = "".join(("A" if c != "A" else "C") if m == "0" else c for c, m in zip(w, mask))
    assert sum(a != b for a, b in zip(w, v)) == 7
    bank = synth.bank_from_strings(["".join(rng.choice("ACGT") for _ in range(40)) + w + "GGGG"])
    hits_masked = _brute.masked_hits([bank.seq(0).decode()], v, mask, 1)
    ox = oracle.Index(bank, stride=1, mask=mask)
    r = ox.search([v.encode()], oracle.Params(stride=1, keep_hits=True, min_hsp_len=18))[0]
    got = sorted((int(h["qpos"]), int(h["seq"]), int(h["pos"])) for h in r.hits)
    assert (0, 0, 40) in got and got == sorted(hits_masked)
