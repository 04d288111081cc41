"""Planted-homolog recovery: the measure behind the sensitivity sweep.

The paper (section "Results quality") reports which share of BLAST's alignments
the method finds, by E-value, and that a lower minimum HSP length raises that
share at weak E-values for little extra time.  Without BLAST or the paper's
data, the synthetic query sets stand in: each planted query is a mutated copy
of a known bank interval, so the truth is known.

A planted query counts as recovered at threshold E when one of its reported
alignments lies in the source sequence, overlaps the source interval
[src_pos, src_pos + src_len) and has an E-value of at most E.  Recovery is
reported per divergence bin and per E-value threshold.  This is bookkeeping over
finished results on the host; it does none of the search's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

# divergence bins (fraction of mutated bases) and E-value thresholds of the tables
DIV_EDGES = (0.0, 0.05, 0.10, 0.15, 0.20, 0.25, 1.0)
E_THRESHOLDS = (1e-35, 1e-15, 1e-10, 1e-5, 1e-2, math.inf)


def _fields(a: np.ndarray):
    """(seq, db_start, db_end, evalue) of a result array: the library's field names or
    the oracle's (seq, ds, de, evalue)."""
    names = a.dtype.names or ()
    if "db_start" in names:
        return a["seq"], a["db_start"], a["db_end"], a["evalue"]
    return a["seq"], a["ds"], a["de"], a["evalue"]


def best_evalue(meta: np.ndarray, results) -> np.ndarray:
    """Per query: the smallest E-value among its alignments that hit its planted source
    (inf when none does, or the query is not planted).  meta is the synthetic query
    table [n, 5] = (is_homolog, src_seq, src_pos, src_len, divergence * 1e6)."""
    meta = np.asarray(meta)
    n = meta.shape[0]
    if len(results) != n:
        raise ValueError(f"{len(results)} result arrays for {n} queries")
    out = np.full(n, math.inf)
    for i in range(n):
        if not meta[i, 0] or len(results[i]) == 0:
            continue
        seq, ds, de, ev = _fields(results[i])
        lo, hi = int(meta[i, 2]), int(meta[i, 2]) + int(meta[i, 3])
        on = (seq.astype(np.int64) == int(meta[i, 1])) & (ds.astype(np.int64) < hi) & (de.astype(np.int64) > lo)
        if on.any():
            out[i] = float(np.min(ev[on]))
    return out


def recovery_table(meta: np.ndarray, results) -> dict:
    """Counts of planted queries and of those recovered, by divergence bin and by
    E-value threshold (all thresholds for each bin)."""
    meta = np.asarray(meta)
    best = best_evalue(meta, results)
    planted = meta[:, 0] != 0
    div = meta[:, 4].astype(np.float64) * 1e-6
    found_any = np.isfinite(best)
    by_div = []
    for lo, hi in zip(DIV_EDGES[:-1], DIV_EDGES[1:]):
        sel = planted & (div >= lo) & (div < hi)
        by_div.append({"div_lo": lo, "div_hi": hi, "planted": int(sel.sum()),
                       "found": [int((sel & found_any & (best <= e)).sum()) for e in E_THRESHOLDS]})
    return {"planted": int(planted.sum()), "found": int((planted & found_any).sum()),
            "evalue_thresholds": [e if math.isfinite(e) else None for e in E_THRESHOLDS],
            "found_at_evalue": [int((planted & found_any & (best <= e)).sum()) for e in E_THRESHOLDS],
            "by_divergence": by_div}
