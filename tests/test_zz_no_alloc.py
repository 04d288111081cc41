"""gn_align_hsps_static: the alignment entry point that allocates no device memory.

It serves callers that cannot allocate on their path (their device memory belongs to
another allocator, or they run too close to a memory limit to risk an allocation
failure).  Its alignments must equal those of gn_search's own alignment phase for the
same HSPs.  This file is collected last on purpose: it runs after every other test
in a full run, and also passes alone in a fresh process."""
import numpy as np
import pytest

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
    return torch, gn, ix, qs, sel, aln


def _run(torch, gn, ix, qs, hsps, scoring):
    dev_q = torch.from_numpy(qs.bases).cuda()
    dev_s = torch.from_numpy(qs.start.view(np.int64)).cuda()
    dev_h = torch.from_numpy(np.ascontiguousarray(hsps).view(np.uint8)).cuda()
    out = torch.full((len(hsps) * gn.HIT_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    gn.gn_align_hsps_static(ix.handle, dev_q.data_ptr(), dev_s.data_ptr(), qs.n, dev_h.data_ptr(), len(hsps),
                            scoring, 16, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
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
