"""Parity of the CUDA path (through the C ABI) with the CPU oracle, phase by phase.

Integer outputs (index, hits, HSPs, alignments, scores, ranks) must be identical;
e-values and bit scores agree to 1e-9 relative (both are fp64: exp and log of the
device and of the host C library may differ in the last bit)."""
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


def assert_ranked_equal(got, exp, ctx=""):
    assert len(got) == len(exp), f"{ctx}: {len(got)} vs {len(exp)} alignments"
    for fg, fe in FIELDS:
        a, b = got[fg].astype(np.int64), exp[fe].astype(np.int64)
        assert np.array_equal(a, b), f"{ctx}: field {fg} differs at {np.nonzero(a != b)[0][:5]}"
    for f in ("evalue", "bits"):
        a, b = got[f], exp[f]
        tiny = (np.abs(a) < 1e-300) & (np.abs(b) < 1e-300)
        ok = tiny | np.isclose(a, b, rtol=1e-9, atol=0)
        assert ok.all(), f"{ctx}: {f} differs"


def by_query(arr, qi):
    return arr[arr["query"] == qi]


def hsp_tuples_gpu(arr):
    return [tuple(int(r[f]) for f in ("seq", "q_start", "q_end", "db_start", "db_end", "len")) for r in arr]


def hsp_tuples_or(arr):
    return [tuple(int(r[f]) for f in ("seq", "qs", "qe", "ds", "de", "len")) for r in arr]


def aln_tuples_gpu(arr):
    return [tuple(int(r[f]) for f in ("seq", "q_start", "q_end", "db_start", "db_end", "score")) for r in arr]


def aln_tuples_or(arr):
    return [tuple(int(r[f]) for f in ("seq", "qs", "qe", "ds", "de", "score")) for r in arr]


def check_stages(g, res, ref, n, ctx):
    hsp = res.stage(g.GN_STAGE_HSP)
    ext = res.stage(g.GN_STAGE_EXT)
    merged = res.stage(g.GN_STAGE_MERGED)
    sel = res.stage(g.GN_STAGE_SELECTED)
    aln = res.stage(g.GN_STAGE_ALIGNED)
    counts = res.stage(g.GN_STAGE_HIT_COUNTS)
    assert len(hsp) == len(ext)
    for i in range(n):
        r = ref[i]
        c = f"{ctx} query {i}"
        assert int(counts[i]) == r.n_hits, c
        h_mask = hsp["query"] == i
        assert sorted(hsp_tuples_gpu(hsp[h_mask])) == sorted(hsp_tuples_or(r.hsp)), c + " HSPs"
        pairs_gpu = sorted(zip(hsp_tuples_gpu(hsp[h_mask]), hsp_tuples_gpu(ext[h_mask])))
        pairs_or = sorted(zip(hsp_tuples_or(r.hsp), hsp_tuples_or(r.ext)))
        assert pairs_gpu == pairs_or, c + " extension"
        assert hsp_tuples_gpu(by_query(merged, i)) == hsp_tuples_or(r.merged), c + " overlap merge"
        assert hsp_tuples_gpu(by_query(sel, i)) == hsp_tuples_or(r.sel), c + " selection"
        assert aln_tuples_gpu(by_query(aln, i)) == aln_tuples_or(r.aln), c + " alignment"
        assert_ranked_equal(res.query(i), r.ranked, c + " ranking")


# ---------------------------------------------------------------- index --
@pytest.mark.parametrize("k,t", [(11, 11), (11, 1), (5, 3), (8, 8), (16, 16)])
def test_index_bitexact_tiny(gn, k, t):
    bank = synth.make_bank("tiny", n_seqs=400 if k < 16 else 1000)
    ix = gn.Index.from_bank(bank, k=k, stride=t)
    got = ix.export() if k <= 12 else None
    ref = oracle.Index(bank, k=k, stride=t)
    assert ix.info().n_postings == ref.n_postings
    if got is not None:
        bs, ps, pp = ref.buckets()
        assert np.array_equal(got[0], bs)
        assert np.array_equal(got[1], ps) and np.array_equal(got[2], pp)


def test_index_bitexact_odd_bank(gn):
    rng = np.random.default_rng(5)
    seqs = []
    for i in range(300):
        L = int(rng.integers(0, 90))
        s = bytearray(rng.choice(list(b"ACGT"), size=L).astype(np.uint8).tobytes())
        if L and i % 4 == 0:
            s[int(rng.integers(L))] = ord("N")
        if L and i % 5 == 0:
            s[int(rng.integers(L))] = ord(rng.choice(list("acgtuU")))
        seqs.append(bytes(s))
    bank = synth.bank_from_strings(seqs)
    for k, t in ((4, 2), (7, 1), (3, 3)):
        ix = gn.Index.from_bank(bank, k=k, stride=t)
        bs, ps, pp = ix.export()
        r = oracle.Index(bank, k=k, stride=t).buckets()
        assert np.array_equal(bs, r[0]) and np.array_equal(ps, r[1]) and np.array_equal(pp, r[2])


@pytest.mark.parametrize("mask,t", [("1101", 4), ("111010010100110111", 18), ("110011", 1), ("1" * 11, 11)])
def test_masked_index_bitexact(gn, mask, t):
    """Spaced seeds: windows of the mask's length keyed by their kept bases."""
    bank = synth.make_bank("tiny", n_seqs=300)
    ix = gn.Index.from_bank(bank, stride=t, mask=mask)
    ref = oracle.Index(bank, stride=t, mask=mask)
    assert ix.info().n_postings == ref.n_postings
    got, exp = ix.export(), ref.buckets()
    assert all(np.array_equal(a, b) for a, b in zip(got, exp))


# --------------------------------------------------------------- search --
@pytest.fixture(scope="module")
def tiny(gn):
    bank = synth.make_bank("tiny")
    qs = synth.make_queries("tiny", bank)
    return bank, qs, gn.Index.from_bank(bank), oracle.Index(bank)


def test_search_stages_tiny(gn, tiny):
    bank, qs, ix, ox = tiny
    flags = gn.GN_FLAG_KEEP_STAGES | gn.GN_FLAG_KEEP_HITS
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=flags))
    ref = ox.search(qs, oracle.Params(keep_hits=True))
    hits = res.stage(gn.GN_STAGE_HITS)
    for i in range(qs.n):
        got = sorted((int(h["qpos"]), int(h["seq"]), int(h["pos"])) for h in hits[hits["query"] == i])
        exp = sorted((int(h["qpos"]), int(h["seq"]), int(h["pos"])) for h in ref[i].hits)
        assert got == exp, f"hits of query {i}"
    check_stages(gn, res, ref, qs.n, "tiny")


@pytest.fixture(scope="module")
def mid_small(gn):
    bank = synth.make_bank("mid", n_seqs=20000)
    q1 = synth.make_queries("mid", bank, n=60)
    q2 = synth.make_queries("batched", bank, n=60)
    qs = synth.queries_from_strings([q1.query(i) for i in range(q1.n)] + [q2.query(i) for i in range(q2.n)])
    return bank, qs, gn.Index.from_bank(bank), oracle.Index(bank)


def test_search_stages_mid_small(gn, mid_small):
    bank, qs, ix, ox = mid_small
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    check_stages(gn, res, ref, qs.n, "mid")
    assert sum(len(r.ranked) for r in ref) > 100


@pytest.mark.parametrize("stride,env", [(1, {}), (4, {}), (1, {"GN_SPILL_ROOM": "64"})])
def test_search_stages_mid_small_stride(gn, mid_small, stride, env, monkeypatch):
    """Index at stride 1 (every window) and 4: D = 3 stride, so chains are short-gapped.  At
    stride 1 most hits pass the repeat filter and many buckets overflow into the spill path."""
    bank, qs, _, _ = mid_small
    for k_, v in env.items():
        monkeypatch.setenv(k_, v)
    sub = qs.subset(range(0, qs.n, 2))
    ix = gn.Index.from_bank(bank, stride=stride)
    ox = oracle.Index(bank, stride=stride)
    res = gn.search(ix, sub.start, sub.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(sub, oracle.Params(stride=stride), threads=os.cpu_count() or 1)
    check_stages(gn, res, ref, sub.n, f"stride {stride}")
    ix.close()


@pytest.mark.parametrize("mask,t", [("111010010100110111", 18), ("111010010100110111", 6)])
def test_search_stages_masked(gn, mid_small, mask, t):
    """The paper's mask: every phase equals the oracle's with spaced seeds."""
    bank, qs, _, _ = mid_small
    sub = qs.subset(range(0, qs.n, 2))
    ix = gn.Index.from_bank(bank, stride=t, mask=mask)
    ox = oracle.Index(bank, stride=t, mask=mask)
    res = gn.search(ix, sub.start, sub.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(sub, oracle.Params(stride=t), threads=os.cpu_count() or 1)
    check_stages(gn, res, ref, sub.n, f"mask {mask} stride {t}")
    assert sum(len(r.ranked) for r in ref) > 50
    ix.close()


def test_both_strands_mid_small(gn, mid_small):
    """GN_FLAG_BOTH_STRANDS: result 2i is query i as given, 2i + 1 its reverse complement."""
    bank, qs, ix, ox = mid_small
    # every third query, plus the reverse complements of two bank stretches (found on strand 2i + 1)
    picked = [qs.query(i) for i in range(0, qs.n, 3)]
    picked += [oracle.reverse_complement(bank.seq(5)[:600]), oracle.reverse_complement(bank.seq(77)[100:900])]
    sub = synth.queries_from_strings(picked)
    res = gn.search(ix, sub.start, sub.bases, params=gn.make_params(flags=gn.GN_FLAG_BOTH_STRANDS))
    assert res.n_queries == 2 * sub.n
    ref = ox.search(sub, oracle.Params(both_strands=True), threads=os.cpu_count() or 1)
    for i in range(2 * sub.n):
        assert_ranked_equal(res.query(i), ref[i].ranked, f"both strands, result {i}")
    plain = gn.search(ix, sub.start, sub.bases)
    for i in range(sub.n):
        a, b = plain.query(i), res.query(2 * i)
        assert np.array_equal(b["query"], np.full(len(b), 2 * i, dtype=b["query"].dtype))
        assert all(np.array_equal(a[f], b[f]) for f in a.dtype.names if f != "query")
    assert sum(len(res.query(2 * i + 1)) for i in range(sub.n)) > 0


def test_batched_equals_plain(gn, mid_small):
    bank, qs, ix, ox = mid_small
    allq = gn.search(ix, qs.start, qs.bases)
    for i in range(0, qs.n, 7):
        one = synth.queries_from_strings([qs.query(i)])
        r1 = gn.search(ix, one.start, one.bases).query(0)
        ra = allq.query(i)
        assert np.array_equal(r1[[f for f, _ in FIELDS]], ra[[f for f, _ in FIELDS]]), i


def test_chunked_equals_unchunked(gn, mid_small, monkeypatch):
    bank, qs, ix, ox = mid_small
    whole = gn.search(ix, qs.start, qs.bases).all()
    monkeypatch.setenv("GN_MAX_CHUNK_HITS", "20000")
    parts = gn.search(ix, qs.start, qs.bases).all()
    for a, b in zip(whole, parts):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("env", [{"GN_HIT_GROUPING": "sort"}, {"GN_BUCKET_CAP": "64"}, {"GN_TILE_FILTER": "0"},
                                 {"GN_RANK_PATH": "sort"}, {"GN_TILE_POS": "64"}, {"GN_SELECT_PATH": "sort"},
                                 {"GN_BUCKET_CAP": "64", "GN_MAX_CHUNK_HITS": "30000"},
                                 {"GN_BUCKET_CAP": "64", "GN_SPILL_ROOM": "16"}, {"GN_SW_LONG_ROWS": "1"},
                                 {"GN_SW_LONG_ROWS": "100"}, {"GN_SW_LANES": "16"}, {"GN_SW_LANES": "32"},
                                 {"GN_BUCKET_TARGET": "2048"}, {"GN_BUCKET_TARGET": "16384"},
                                 {"GN_XDROP_LANE_STEPS": "0"}, {"GN_XDROP_LANE_STEPS": "5"},
                                 {"GN_XDROP_LANE_STEPS": "100000"}, {"GN_SORT_THREE_KERNEL": "1"}])
def test_hit_grouping_paths_agree_with_oracle(gn, mid_small, monkeypatch, env):
    """The global sort path, the bucketed path and its overflow fallback give the oracle's HSPs."""
    bank, qs, ix, ox = mid_small
    for k_, v in env.items():
        monkeypatch.setenv(k_, v)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    check_stages(gn, res, ref, qs.n, str(env))


def test_device_queries_equal_host_queries(gn, mid_small):
    import torch
    bank, qs, ix, ox = mid_small
    a = gn.search(ix, qs.start, qs.bases).all()
    b = gn.search(ix, qs.start, torch.from_numpy(qs.bases).cuda()).all()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("kw", [dict(max_alignments=0), dict(max_alignments=1), dict(band_w=0),
                                dict(band_w=20), dict(band_w=64), dict(band_w=128), dict(band_w=150),
                                dict(xdrop=5), dict(max_hit_distance=11, min_hsp_len=33),
                                dict(min_hsp_len=11), dict(min_hsp_len=5)])
def test_parameters_mid_small(gn, mid_small, kw):
    bank, qs, ix, ox = mid_small
    sub = qs.subset(range(0, qs.n, 3))
    res = gn.search(ix, sub.start, sub.bases, params=gn.make_params(**kw))
    okw = {("max_alignments" if k == "max_alignments" else k): v for k, v in kw.items()}
    ref = ox.search(sub, oracle.Params(**okw), threads=os.cpu_count() or 1)
    for i in range(sub.n):
        assert_ranked_equal(res.query(i), ref[i].ranked, f"{kw} query {i}")


def test_edge_queries(gn, tiny):
    bank, qs, ix, ox = tiny
    empty = synth.queries_from_strings([])
    r = gn.search(ix, empty.start, empty.bases)
    assert r.n_queries == 0
    src = bank.seq(17)
    cases = [b"", b"ACG", b"N" * 50, src[:300], src[:150] + b"NNNN" + src[154:400], src[:300].lower(),
             b"ACGTACGTACG"]
    q = synth.queries_from_strings(cases)
    res = gn.search(ix, q.start, q.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(q, oracle.Params())
    check_stages(gn, res, ref, q.n, "edge")
    assert len(res.query(3)) >= 1 and int(res.query(3)[0]["seq"]) == 17


def test_too_long_query_rejected(gn, tiny):
    bank, qs, ix, ox = tiny
    q = synth.queries_from_strings([b"A" * 70000])
    srv = gn.Server(ix, 1 << 30)
    with pytest.raises(gn.GnError) as e:  # the request loop takes queries of one segment
        srv.submit(q.query(0))
    assert e.value.status == gn.GN_ETOOBIG
    srv.stop()
    assert gn.search(ix, q.start, q.bases).n_queries == 1  # gn_search takes it in segments


def test_autotune(gn, mid_small):
    """The autotuner picks a band width from the calibration sample and a result-invariant
    kernel tuning; results with the tuning installed equal the untuned ones, and results with
    the chosen band equal the oracle's with that band."""
    bank, qs, _, ox = mid_small
    ix = gn.Index.from_bank(bank)
    sub = qs.subset(range(0, qs.n, 4))
    before = gn.search(ix, sub.start, sub.bases).all()
    p, tuning = gn.autotune(ix, sub.start, sub.bases)
    assert p.band_w in (16, 32, 64, 128)
    assert tuning["fill_threads"] in (256, 512) and tuning["tile_hits"] in (25000, 50000, 100000)
    assert tuning["bucket_target"] in (2048, 4096, 8192)
    assert tuning["sw_lanes"] in (8, 16, 32) and tuning["sw_wave_rows"] in (256, 512, 1024)
    assert gn.get_tuning(ix) == tuning
    after = gn.search(ix, sub.start, sub.bases).all()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    res = gn.search(ix, sub.start, sub.bases, params=p)
    ref = ox.search(sub, oracle.Params(band_w=p.band_w), threads=os.cpu_count() or 1)
    for i in range(sub.n):
        assert_ranked_equal(res.query(i), ref[i].ranked, f"autotuned band {p.band_w} query {i}")
    # twice the chosen band raises the sample's total score by at most 0.5 % (unless it is the widest)
    if p.band_w < 128:
        wide = gn.search(ix, sub.start, sub.bases, params=gn.make_params(band_w=2 * p.band_w)).all()
        a = sum(int(x["score"].sum()) for x in res.all())
        b = sum(int(x["score"].sum()) for x in wide)
        assert b - a <= 0.005 * max(a, 1)
    gn.set_tuning(ix)
    assert gn.get_tuning(ix) == {"tile_hits": 0, "fill_threads": 0, "bucket_target": 0, "sw_lanes": 0,
                                 "sw_wave_rows": 0}
    ix.close()


@pytest.mark.parametrize("kw", [dict(), dict(min_hsp_len=11), dict(max_hit_distance=66, xdrop=40)])
def test_sensitivity_recovery_matches_oracle(gn, mid_small, kw):
    from paper_1507_02987_gb300.sensitivity import recovery_table
    bank, _, ix, ox = mid_small
    qs = synth.make_queries("mid", bank, n=60)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(**kw)).all()
    ref = [r.ranked for r in ox.search(qs, oracle.Params(**kw), threads=os.cpu_count() or 1)]
    got, exp = recovery_table(qs.meta, res), recovery_table(qs.meta, ref)
    assert got == exp and got["planted"] == qs.n and got["found"] > qs.n // 2


@pytest.mark.parametrize("band_w", [0, 1, 16, 20, 24])
def test_wavefront_alignment_path(gn, mid_small, band_w, monkeypatch):
    """Every alignment through the anti-diagonal path (bands up to 64 diagonals) gives the oracle's."""
    bank, qs, ix, ox = mid_small
    monkeypatch.setenv("GN_SW_LONG_ROWS", "1")
    sub = qs.subset(range(0, qs.n, 2))
    res = gn.search(ix, sub.start, sub.bases, params=gn.make_params(band_w=band_w))
    ref = ox.search(sub, oracle.Params(band_w=band_w), threads=os.cpu_count() or 1)
    for i in range(sub.n):
        assert_ranked_equal(res.query(i), ref[i].ranked, f"band {band_w} query {i}")


@pytest.mark.parametrize("stride", [11, 1])
def test_tandem_repeats_equal_qs_groups(gn, stride):
    """Tandem repeats of a unit whose length is a multiple of the stride: one query stretch
    hits every copy with the same window phase, so the extended HSPs of many diagonals start
    at the same query position.  The overlap merge takes such records by (ds, qe); every
    phase, and the merged order, equals the oracle's."""
    rng = np.random.default_rng(17)
    alphabet = np.frombuffer(b"ACGT", dtype=np.uint8)
    rand = lambda n: alphabet[rng.integers(0, 4, n)].tobytes()
    unit = rand(66)
    seqs, queries = [], []
    for i in range(40):
        copies = int(rng.integers(3, 9))
        body = bytearray(unit * copies)
        for _ in range(int(rng.integers(0, 4))):  # a few point changes between copies
            body[int(rng.integers(len(body)))] = int(alphabet[rng.integers(0, 4)])
        seqs.append(rand(int(rng.integers(0, 200))) + bytes(body) + rand(int(rng.integers(0, 200))))
    seqs += [rand(int(rng.integers(100, 900))) for _ in range(200)]
    bank = synth.bank_from_strings(seqs)
    for j in range(12):
        n_units = int(rng.integers(1, 4))
        q = bytearray(rand(int(rng.integers(0, 40))) + unit * n_units + rand(int(rng.integers(0, 40))))
        if j % 3 == 0:
            q[int(rng.integers(len(q)))] = ord("T")
        queries.append(bytes(q))
    qs = synth.queries_from_strings(queries)
    ix = gn.Index.from_bank(bank, stride=stride)
    ox = oracle.Index(bank, stride=stride)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    ref = ox.search(qs, oracle.Params(stride=stride), threads=os.cpu_count() or 1)
    check_stages(gn, res, ref, qs.n, f"tandem repeats, stride {stride}")
    ext = res.stage(gn.GN_STAGE_EXT)
    keys = {}
    for r in ext:
        keys[(int(r["query"]), int(r["seq"]), int(r["q_start"]))] = keys.get(
            (int(r["query"]), int(r["seq"]), int(r["q_start"])), 0) + 1
    assert max(keys.values()) >= 3  # groups of equal (query, sequence, qs) did occur
    ix.close()


def test_extension_reaches_both_array_starts(gn):
    """A left extension that runs to position 0 of the packed query array and of the packed
    bank at once (its last 16-base window starts before both arrays), and a right extension
    that runs to the end of both: every phase equals the oracle's."""
    rng = np.random.default_rng(23)
    alphabet = np.frombuffer(b"ACGT", dtype=np.uint8)
    rand = lambda n: alphabet[rng.integers(0, 4, n)].tobytes()
    q = bytearray(rand(700))
    head = bytearray(q)
    head[10] = ord("A") if head[10] != ord("A") else ord("C")  # the bank window at 0 misses; the HSP starts at 11
    tail = bytearray(q[-300:])
    tail[-5] = ord("G") if tail[-5] != ord("G") else ord("T")
    seqs = [bytes(head)] + [rand(int(rng.integers(200, 900))) for _ in range(150)] + [bytes(tail)]
    bank = synth.bank_from_strings(seqs)
    qs = synth.queries_from_strings([bytes(q), bytes(q[-300:])])
    for stride in (11, 4):
        ix = gn.Index.from_bank(bank, stride=stride)
        ox = oracle.Index(bank, stride=stride)
        res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
        ref = ox.search(qs, oracle.Params(stride=stride), threads=os.cpu_count() or 1)
        check_stages(gn, res, ref, qs.n, f"array starts, stride {stride}")
        ext = res.stage(gn.GN_STAGE_EXT)
        first = ext[(ext["query"] == 0) & (ext["seq"] == 0)]
        assert len(first) and int(first["q_start"].min()) == 0 and int(first["db_start"].min()) == 0
        ix.close()
