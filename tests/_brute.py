"""Brute-force and textbook references used to pin the oracle on tiny inputs.

These are deliberately different formulations from the oracle's: string
comparison instead of 2-bit codes, dictionaries instead of sorting, explicit
enumeration of alignments or a suffix recursion instead of Gotoh's matrices.
"""
from __future__ import annotations

import functools
import itertools

ACGT = "ACGT"


def is_base(c: str) -> bool:
    return c in "ACGTUacgtu"


def norm(c: str) -> str:
    c = c.upper()
    return "T" if c == "U" else c


def bank_windows(seqs, k, t):
    """{window string: [(seq, pos), ...]} over non-overlapping windows (pos = 0, t, 2t, ...)."""
    d = {}
    for s, seq in enumerate(seqs):
        for pos in range(0, len(seq) - k + 1, t):
            w = seq[pos:pos + k]
            if all(is_base(c) for c in w):
                d.setdefault("".join(norm(c) for c in w), []).append((s, pos))
    return d


def hits(seqs, query, k, t):
    """Every (qpos, seq, pos) with equal k-base strings (query window at every offset)."""
    out = []
    for s, seq in enumerate(seqs):
        for pos in range(0, len(seq) - k + 1, t):
            w = seq[pos:pos + k]
            if not all(is_base(c) for c in w):
                continue
            w = "".join(norm(c) for c in w)
            for qpos in range(0, len(query) - k + 1):
                v = query[qpos:qpos + k]
                if all(is_base(c) for c in v) and "".join(norm(c) for c in v) == w:
                    out.append((qpos, s, pos))
    return out


def chains(hit_list, k, D, min_len):
    """HSPs from hits: same (seq, diagonal) and query gaps <= D; kept if length >= min_len."""
    groups = {}
    for qpos, s, pos in hit_list:
        groups.setdefault((s, pos - qpos), []).append(qpos)
    out = []
    for (s, d), qs in groups.items():
        qs.sort()
        run = [qs[0]]
        for x in qs[1:] + [None]:
            if x is not None and x - run[-1] <= D:
                run.append(x)
                continue
            a, b = run[0], run[-1] + k
            if b - a >= min_len:
                out.append((s, a, b, a + d, b + d, b - a))
            if x is not None:
                run = [x]
    return sorted(out)


def pair(a: str, b: str, match: int, mismatch: int) -> int:
    return match if (is_base(a) and is_base(b) and norm(a) == norm(b)) else mismatch


def enumerate_global(a: str, b: str):
    """All global alignments of a and b as column strings over {'M','I','D'}:
    M = a[i] with b[j], I = a[i] against a gap, D = b[j] against a gap."""
    def rec(i, j):
        if i == len(a) and j == len(b):
            yield ""
            return
        if i < len(a) and j < len(b):
            for r in rec(i + 1, j + 1):
                yield "M" + r
        if i < len(a):
            for r in rec(i + 1, j):
                yield "I" + r
        if j < len(b):
            for r in rec(i, j + 1):
                yield "D" + r
    return rec(0, 0)


def score_columns(a: str, b: str, cols: str, match, mismatch, gap_open, gap_extend) -> int:
    """Score of one alignment written as columns; a gap run of length g scores gap_open + g*gap_extend."""
    i = j = 0
    total = 0
    prev = None
    for c in cols:
        if c == "M":
            total += pair(a[i], b[j], match, mismatch)
            i += 1
            j += 1
        else:
            total += gap_extend + (gap_open if c != prev else 0)
            if c == "I":
                i += 1
            else:
                j += 1
        prev = c
    return total


def local_score_enumerated(a: str, b: str, match=1, mismatch=-3, gap_open=-5, gap_extend=-2) -> int:
    """Best local alignment score by enumerating every pair of substrings and every alignment."""
    best = 0
    for i0, i1 in itertools.combinations(range(len(a) + 1), 2):
        for j0, j1 in itertools.combinations(range(len(b) + 1), 2):
            sa, sb = a[i0:i1], b[j0:j1]
            for cols in enumerate_global(sa, sb):
                best = max(best, score_columns(sa, sb, cols, match, mismatch, gap_open, gap_extend))
    return best


def global_score(a: str, b: str, match=1, mismatch=-3, gap_open=-5, gap_extend=-2, diag_range=None,
                 offset=(0, 0)) -> int:
    """Best end-to-end alignment score of a and b (suffix recursion on (i, j, previous column)).
    diag_range=(lo, hi) restricts aligned/visited cells to lo <= (j+oj) - (i+oi) <= hi, with the
    offsets giving the absolute coordinates of a[0] and b[0]."""
    import sys
    sys.setrecursionlimit(100000)
    NEG = -10 ** 9
    oi, oj = offset

    def ok(i, j):
        if diag_range is None:
            return True
        d = (j + oj) - (i + oi)
        return diag_range[0] <= d <= diag_range[1]

    @functools.lru_cache(maxsize=None)
    def f(i, j, prev):
        if i == len(a) and j == len(b):
            return 0
        best = NEG
        if i < len(a) and j < len(b) and ok(i, j):
            best = max(best, pair(a[i], b[j], match, mismatch) + f(i + 1, j + 1, "M"))
        if i < len(a) and ok(i, j - 1 if j > 0 else j):
            best = max(best, gap_extend + (gap_open if prev != "I" else 0) + f(i + 1, j, "I"))
        if j < len(b) and ok(i - 1 if i > 0 else i, j):
            best = max(best, gap_extend + (gap_open if prev != "D" else 0) + f(i, j + 1, "D"))
        return best

    r = f(0, 0, None)
    f.cache_clear()
    return r


def kadane(scores) -> int:
    best = cur = 0
    for s in scores:
        cur = max(0, cur + s)
        best = max(best, cur)
    return best


def kept(w: str, mask: str) -> str:
    """The bases of window w at the mask's '1' positions, normalised."""
    return "".join(norm(c) for c, m in zip(w, mask) if m == "1")


def masked_windows(seqs, mask, t):
    """{kept-base string: [(seq, pos), ...]} over windows of len(mask) at pos = 0, t, 2t, ...;
    a window with a non-base at a kept position is not indexed."""
    span = len(mask)
    d = {}
    for s, seq in enumerate(seqs):
        for pos in range(0, len(seq) - span + 1, t):
            w = seq[pos:pos + span]
            if all(is_base(c) for c, m in zip(w, mask) if m == "1"):
                d.setdefault(kept(w, mask), []).append((s, pos))
    return d


def masked_hits(seqs, query, mask, t):
    """Every (qpos, seq, pos) whose query window and bank window agree at the kept positions."""
    span = len(mask)
    out = []
    for s, seq in enumerate(seqs):
        for pos in range(0, len(seq) - span + 1, t):
            w = seq[pos:pos + span]
            if not all(is_base(c) for c, m in zip(w, mask) if m == "1"):
                continue
            for qpos in range(0, len(query) - span + 1):
                v = query[qpos:qpos + span]
                if all(is_base(c) for c, m in zip(v, mask) if m == "1") and kept(v, mask) == kept(w, mask):
                    out.append((qpos, s, pos))
    return out
