"""Planted-homolog recovery (the sensitivity sweep's measure), on the CPU.

Hand-made result tables pin the rule (same sequence, overlapping interval,
E-value at most the threshold); the oracle pins what the method does with it: a
lower minimum HSP length never loses a planted homolog that the default finds."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1507_02987_gb300 import HIT_DTYPE
from paper_1507_02987_gb300.sensitivity import E_THRESHOLDS, best_evalue, recovery_table

ORACLE_DTYPE = np.dtype([("seq", "<u4"), ("ds", "<u4"), ("de", "<u4"), ("evalue", "<f8")])


def _rows(dtype, rows):
    a = np.zeros(len(rows), dtype=dtype)
    names = ("seq", "db_start", "db_end", "evalue") if "db_start" in dtype.names else ("seq", "ds", "de", "evalue")
    for i, r in enumerate(rows):
        for n, v in zip(names, r):
            a[i][n] = v
    return a


@pytest.mark.parametrize("dtype", [HIT_DTYPE, ORACLE_DTYPE])
def test_recovery_rule_hand_cases(dtype):
    # meta rows: is_homolog, src_seq, src_pos, src_len, divergence * 1e6
    meta = np.array([[1, 5, 100, 200, 30000],     # found twice, best 1e-40
                     [1, 5, 100, 200, 70000],     # touches the interval's end / wrong sequence: missed
                     [0, 0, 0, 10, 0],            # not planted: never counted
                     [1, 2, 0, 50, 220000],       # found at a weak E-value only
                     [1, 3, 10, 20, 120000]],     # no alignments
                    dtype=np.uint64)
    results = [_rows(dtype, [(5, 299, 400, 1e-20), (5, 50, 120, 1e-40), (4, 100, 300, 1e-90)]),
               _rows(dtype, [(5, 300, 500, 1e-50), (5, 0, 100, 1e-50), (6, 100, 300, 1e-50)]),
               _rows(dtype, [(0, 0, 10, 1e-60)]),
               _rows(dtype, [(2, 0, 50, 5.0)]),
               _rows(dtype, [])]
    best = best_evalue(meta, results)
    assert best[0] == 1e-40 and best[3] == 5.0
    assert math.isinf(best[1]) and math.isinf(best[2]) and math.isinf(best[4])
    t = recovery_table(meta, results)
    assert t["planted"] == 4 and t["found"] == 2
    assert len(t["found_at_evalue"]) == len(E_THRESHOLDS)
    assert t["found_at_evalue"] == [1, 1, 1, 1, 1, 2]
    bins = {(b["div_lo"], b["div_hi"]): (b["planted"], b["found"]) for b in t["by_divergence"]}
    assert bins[(0.0, 0.05)] == (1, [1] * 6)
    assert bins[(0.05, 0.10)] == (1, [0] * 6)
    assert bins[(0.10, 0.15)] == (1, [0] * 6)
    assert bins[(0.20, 0.25)] == (1, [0, 0, 0, 0, 0, 1])
    assert sum(b["planted"] for b in t["by_divergence"]) == 4


def test_recovery_rejects_mismatched_lengths():
    with pytest.raises(ValueError):
        best_evalue(np.zeros((2, 5), dtype=np.uint64), [np.zeros(0, dtype=HIT_DTYPE)])


def test_lower_min_hsp_len_never_loses_a_homolog():
    bank = synth.make_bank("mid", n_seqs=20000)
    qs = synth.make_queries("mid", bank, n=40)
    ix = oracle.Index(bank)
    tables, best = {}, {}
    for m in (22, 16, 11):
        res = ix.search(qs, oracle.Params(min_hsp_len=m), threads=os.cpu_count() or 1)
        ranked = [r.ranked for r in res]
        tables[m] = recovery_table(qs.meta, ranked)
        best[m] = best_evalue(qs.meta, ranked)
    assert tables[22]["planted"] == qs.n
    assert tables[22]["found"] >= qs.n // 2  # 2-25 % divergence: most are found at the default
    for lo, hi in ((22, 16), (16, 11)):
        # a homolog found with longer HSPs is found with shorter ones too (the top-N cut
        # keeps the longest, and the longer HSPs are still among the candidates)
        assert (np.isinf(best[lo]) | np.isfinite(best[hi])).all(), (lo, hi)
        assert tables[hi]["found"] >= tables[lo]["found"]
