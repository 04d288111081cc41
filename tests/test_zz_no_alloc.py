"""gn_align_hsps_static: the alignment entry point that allocates no device memory.

It serves callers that cannot allocate on their path (their device memory belongs to
another allocator, or they run too close to a memory limit to risk an allocation
failure).  Its alignments must equal those of gn_search's own alignment phase for the
same HSPs.  This file is collected last on purpose: it runs after every other test
in a full run, and also passes alone in a fresh process."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("query", "seq", "q_start", "q_end", "db_start", "db_end", "score")


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_02987_gb300 import _build
    _build.build()
    import paper_1507_02987_gb300 as gn
    bank = synth.make_bank("mid", n_seqs=3000)
    tq = synth.make_queries("mid", bank, n=25)
    bq = synth.make_queries("batched", bank, n=25)
    qs = synth.queries_from_strings([tq.query(i) for i in range(tq.n)] + [bq.query(i) for i in range(bq.n)])
    ix = gn.Index.from_bank(bank)
    res = gn.search(ix, qs.start, qs.bases, params=gn.make_params(flags=gn.GN_FLAG_KEEP_STAGES))
    sel = res.stage(gn.GN_STAGE_SELECTED)
    aln = res.stage(gn.GN_STAGE_ALIGNED)
    assert len(sel) == len(aln) and len(sel) > 20
    _setup.bank = bank
    return torch, gn, ix, qs, sel, aln


def _run(torch, gn, ix, qs, hsps, scoring, band_w=16):
    dev_q = torch.from_numpy(qs.bases).cuda()
    dev_s = torch.from_numpy(qs.start.view(np.int64)).cuda()
    dev_h = torch.from_numpy(np.ascontiguousarray(hsps).view(np.uint8)).cuda()
    out = torch.full((len(hsps) * gn.HIT_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    gn.gn_align_hsps_static(ix.handle, dev_q.data_ptr(), dev_s.data_ptr(), qs.n, dev_h.data_ptr(), len(hsps),
                            scoring, band_w, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    free_after = torch.cuda.mem_get_info()[0]
    got = np.frombuffer(out.cpu().numpy().tobytes(), dtype=gn.HIT_DTYPE)
    return got, free_before, free_after


def test_static_alignment_equals_search_alignment_phase_twice():
    torch, gn, ix, qs, sel, aln = _setup()
    sc = gn.make_scoring()
    # first call: every selected HSP of the search
    got1, _, _ = _run(torch, gn, ix, qs, sel, sc)
    for f in FIELDS:
        assert np.array_equal(got1[f], aln[f]), f
    # second call in a row: a different set (every other HSP, reversed), reusing the same scratch
    idx = np.arange(len(sel))[::-2]
    got2, fb, fa = _run(torch, gn, ix, qs, sel[idx], sc)
    for f in FIELDS:
        assert np.array_equal(got2[f], aln[idx][f]), f
    # no device memory was taken by the call
    assert fa == fb


def test_static_alignment_rejects_bad_input():
    torch, gn, ix, qs, sel, aln = _setup()
    bad = sel[:4].copy()
    bad["query"][1] = qs.n + 7
    with pytest.raises(gn.GnError) as e:
        _run(torch, gn, ix, qs, bad, gn.make_scoring())
    assert e.value.status == gn.GN_EINVAL
    with pytest.raises(gn.GnError) as e:
        gn.gn_align_hsps_static(ix.handle, 0, 0, qs.n, 0, 0, gn.make_scoring(), 600, 0)
    assert e.value.status == gn.GN_ETOOBIG


@pytest.mark.parametrize("w", [128, 500])
def test_static_alignment_wide_bands_equal_oracle(w):
    """Bands over 64 diagonals go through the kernel's 32-offset chunks with the horizontal-gap
    carry between chunks; with w = 500 a band spans up to 1,024 diagonals (the scratch's
    limit).  Every alignment equals the oracle's banded Smith-Waterman of the same HSP."""
    torch, gn, ix, qs, sel, aln = _setup()
    bank = _setup.bank
    spread = np.abs((sel["db_start"].astype(np.int64) - sel["q_start"]) - (sel["db_end"].astype(np.int64) - sel["q_end"]))
    hsps = sel[spread + 2 * w + 1 <= 1024][:40]
    assert len(hsps) >= 20
    got, _, _ = _run(torch, gn, ix, qs, hsps, gn.make_scoring(), band_w=w)
    p = oracle.Params(band_w=w)
    for r, h in zip(got, hsps):
        q = qs.query(int(h["query"]))
        s0, s1 = int(bank.seq_start[h["seq"]]), int(bank.seq_start[h["seq"] + 1])
        exp = oracle.banded_sw(q, bank.bases[s0:s1].tobytes(),
                               (int(h["q_start"]), int(h["q_end"]), int(h["db_start"]), int(h["db_end"])), p)
        assert (int(r["score"]), int(r["q_start"]), int(r["q_end"]), int(r["db_start"]), int(r["db_end"])) == exp
        assert int(r["query"]) == int(h["query"]) and int(r["seq"]) == int(h["seq"])


def test_static_alignment_row_limit():
    """A DP window of more than 65,535 rows (a 70,000-base query) is refused with GN_ETOOBIG
    and its record is written with score 0."""
    torch, gn, ix, qs, sel, aln = _setup()
    rng = np.random.default_rng(5)
    long_q = synth.queries_from_strings([bytes(rng.choice(list(b"ACGT"), 70000).astype(np.uint8))])
    h = sel[:1].copy()
    h["query"], h["q_start"], h["q_end"] = 0, 0, 70000
    h["db_start"], h["db_end"] = 0, 70000
    with pytest.raises(gn.GnError) as e:
        _run(torch, gn, ix, long_q, h, gn.make_scoring())
    assert e.value.status == gn.GN_ETOOBIG
