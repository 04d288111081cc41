"""CPU oracle for the Genoogle search path (arXiv 1507.02987).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it shares no code with the CUDA path.  The arithmetic lives in plain C
(``oracle.c``); this module only compiles it and marshals arguments.

Function-to-paper map (section names of the paper):
  build_index        "Inverted Indexes"            bank windows -> (seq, pos) buckets
  search             "Searching process"           the seven phases, per query
  extend             phase 3 (HSP extension with drop-off)
  merge_overlaps     phase 4 (merging overlapped HSPs)
  banded_sw          phase 6 (Smith-Waterman restricted to the HSP's diagonals)
  evalue / bits      phase 7 ("e-value, score, normalized score"; Karlin-Altschul)

Parity is pinned for every function by the tests in ``tests/test_oracle_*.py``
(brute force on tiny inputs, hand-computed cases, closed forms, the paper's
worked index-size example).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgn_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


HIT_DTYPE = np.dtype([("qpos", "<u4"), ("seq", "<u4"), ("pos", "<u4")])
HSP_DTYPE = np.dtype([("seq", "<u4"), ("qs", "<u4"), ("qe", "<u4"), ("ds", "<u4"), ("de", "<u4"),
                      ("len", "<u4")])
ALN_DTYPE = np.dtype([("seq", "<u4"), ("qs", "<u4"), ("qe", "<u4"), ("ds", "<u4"), ("de", "<u4"),
                      ("score", "<i4"), ("rank", "<u4"), ("pad", "<u4"), ("evalue", "<f8"), ("bits", "<f8")])


class _Params(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("lam", ctypes.c_double), ("K", ctypes.c_double),
                ("max_hit_distance", ctypes.c_uint32), ("min_hsp_len", ctypes.c_uint32),
                ("xdrop", ctypes.c_int32), ("max_alignments", ctypes.c_uint32), ("band_w", ctypes.c_uint32),
                ("max_evalue", ctypes.c_double), ("keep_hits", ctypes.c_int32)]


class _Hsp(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("seq", "qs", "qe", "ds", "de", "len")]


class _Aln(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint32), ("qs", ctypes.c_uint32), ("qe", ctypes.c_uint32),
                ("ds", ctypes.c_uint32), ("de", ctypes.c_uint32), ("score", ctypes.c_int32),
                ("rank", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("evalue", ctypes.c_double),
                ("bits", ctypes.c_double)]


class _Result(ctypes.Structure):
    _fields_ = [("n_hits", ctypes.c_uint64), ("hits", ctypes.c_void_p), ("n_hits_kept", ctypes.c_uint64),
                ("hsp", ctypes.c_void_p), ("n_hsp", ctypes.c_uint32),
                ("ext", ctypes.c_void_p), ("n_ext", ctypes.c_uint32),
                ("merged", ctypes.c_void_p), ("n_merged", ctypes.c_uint32),
                ("sel", ctypes.c_void_p), ("n_sel", ctypes.c_uint32),
                ("aln", ctypes.c_void_p), ("n_aln", ctypes.c_uint32),
                ("ranked", ctypes.c_void_p), ("n_ranked", ctypes.c_uint32),
                ("status", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
            lib.or_index_build.restype = vp
            lib.or_index_build.argtypes = [vp, vp, u32, ctypes.c_int, ctypes.c_int]
            lib.or_index_build_masked.restype = vp
            lib.or_index_build_masked.argtypes = [vp, vp, u32, ctypes.c_char_p, ctypes.c_int]
            lib.or_index_build_restricted.restype = vp
            lib.or_index_build_restricted.argtypes = [vp, vp, u32, ctypes.c_char_p, ctypes.c_int, vp, ctypes.c_int]
            lib.or_mark_query_codes.argtypes = [vp, u32, ctypes.c_char_p, vp]
            lib.or_index_free.argtypes = [vp]
            lib.or_index_n_postings.restype = u64
            lib.or_index_n_postings.argtypes = [vp]
            for f in ("or_index_bucket_start", "or_index_post_seq", "or_index_post_pos"):
                getattr(lib, f).restype = vp
                getattr(lib, f).argtypes = [vp]
            lib.or_search_one.restype = ctypes.c_int
            lib.or_search_one.argtypes = [vp, vp, u32, ctypes.POINTER(_Params), ctypes.POINTER(_Result)]
            lib.or_search_batch.restype = ctypes.c_int
            lib.or_search_batch.argtypes = [vp, vp, vp, u32, ctypes.POINTER(_Params), ctypes.c_int, vp]
            lib.or_result_free.argtypes = [ctypes.POINTER(_Result)]
            lib.or_result_free_batch.argtypes = [vp, u32]
            lib.or_extend.argtypes = [vp, u32, vp, u32, ctypes.POINTER(_Params), ctypes.POINTER(_Hsp)]
            lib.or_banded_sw.argtypes = [vp, u32, vp, u32, ctypes.POINTER(_Hsp), ctypes.POINTER(_Params),
                                         ctypes.POINTER(_Aln)]
            lib.or_merge_overlaps.restype = u32
            lib.or_merge_overlaps.argtypes = [vp, u32, vp]
            lib.or_evalue.restype = ctypes.c_double
            lib.or_evalue.argtypes = [i32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Params)]
            lib.or_bits.restype = ctypes.c_double
            lib.or_bits.argtypes = [i32, ctypes.POINTER(_Params)]
            lib.or_rank.restype = u32
            lib.or_rank.argtypes = [vp, u32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Params), vp]
            lib.or_sizeof_result.restype = ctypes.c_size_t
            assert lib.or_sizeof_result() == ctypes.sizeof(_Result)
            _lib = lib
    return _lib


def ungapped_lambda(match: int = 1, mismatch: int = -3) -> float:
    """lambda solving sum_ab p_a p_b exp(lambda s_ab) = 1 for uniform bases (1/4 match, 3/4 mismatch)."""
    f = lambda lam: 0.25 * math.exp(lam * match) + 0.75 * math.exp(lam * mismatch) - 1.0
    lo, hi = 1e-6, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


@dataclass
class Params:
    """Run-time parameters ("Methods", parameters paragraph) plus scoring."""
    k: int = 11
    stride: int = 11
    match: int = 1
    mismatch: int = -3
    gap_open: int = -5
    gap_extend: int = -2
    lam: float = 1.3740631
    K: float = 0.711
    max_hit_distance: int = 0     # 0 -> 3 * stride
    min_hsp_len: int = 0          # 0 -> 2 * k
    xdrop: int = 20
    max_alignments: int = 100     # 0 -> all
    band_w: int = 16
    max_evalue: float = math.inf
    keep_hits: bool = False
    both_strands: bool = False    # also search each query's reverse complement (result 2i + 1)

    def resolved(self) -> "Params":
        import dataclasses
        p = dataclasses.replace(self)
        if p.max_hit_distance == 0:
            p.max_hit_distance = 3 * p.stride
        if p.min_hsp_len == 0:
            p.min_hsp_len = 2 * p.k
        return p

    def _c(self) -> _Params:
        p = self.resolved()
        return _Params(p.match, p.mismatch, p.gap_open, p.gap_extend, p.lam, p.K, p.max_hit_distance,
                       p.min_hsp_len, p.xdrop, p.max_alignments, p.band_w, p.max_evalue, int(p.keep_hits))


def _arr(ptr, n, dtype):
    if n == 0 or not ptr:
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (n * dtype.itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype).copy()


@dataclass
class QueryResult:
    n_hits: int
    hits: np.ndarray      # HIT_DTYPE, sorted by (seq, diagonal, qpos); empty unless keep_hits
    hsp: np.ndarray       # HSP_DTYPE
    ext: np.ndarray
    merged: np.ndarray
    sel: np.ndarray
    aln: np.ndarray       # ALN_DTYPE
    ranked: np.ndarray    # ALN_DTYPE


def _convert(r: _Result) -> QueryResult:
    return QueryResult(int(r.n_hits), _arr(r.hits, int(r.n_hits_kept), HIT_DTYPE),
                       _arr(r.hsp, r.n_hsp, HSP_DTYPE), _arr(r.ext, r.n_ext, HSP_DTYPE),
                       _arr(r.merged, r.n_merged, HSP_DTYPE), _arr(r.sel, r.n_sel, HSP_DTYPE),
                       _arr(r.aln, r.n_aln, ALN_DTYPE), _arr(r.ranked, r.n_ranked, ALN_DTYPE))


class Index:
    """The oracle's inverted index: 4^k buckets of (sequence id, position) pairs."""

    def __init__(self, bank, k: int = 11, stride: int = 11, mask: str | None = None, restrict_to=None,
                 threads: int = 1):
        """k-base windows, or with ``mask`` (e.g. "111010010100110111") windows of the mask's
        length indexed under their kept bases ("Methods"); k is then the mask's weight.

        ``restrict_to`` (a query set) keeps only the buckets of those queries' seed codes, each
        exactly as in the full index, so that searching those queries gives the full index's
        results; the bank is then scanned by ``threads`` threads.  For banks whose full index
        would not fit the host."""
        self._lib = _load()
        self.bank = bank
        self._bases = np.ascontiguousarray(bank.bases, dtype=np.uint8)
        self._start = np.ascontiguousarray(bank.seq_start, dtype=np.uint64)
        if restrict_to is not None:
            m = mask if mask is not None else "1" * k
            k = m.count("1")
            keep = np.zeros(1 << (2 * k), dtype=np.uint8)
            for i in range(restrict_to.n):
                q = np.frombuffer(restrict_to.query(i), dtype=np.uint8)
                self._lib.or_mark_query_codes(q.ctypes.data, len(q), m.encode(), keep.ctypes.data)
            self._h = self._lib.or_index_build_restricted(self._bases.ctypes.data, self._start.ctypes.data,
                                                          bank.n_seqs, m.encode(), stride, keep.ctypes.data,
                                                          max(1, int(threads)))
        elif mask is not None:
            k = mask.count("1")
            self._h = self._lib.or_index_build_masked(self._bases.ctypes.data, self._start.ctypes.data, bank.n_seqs,
                                                      mask.encode(), stride)
        else:
            self._h = self._lib.or_index_build(self._bases.ctypes.data, self._start.ctypes.data, bank.n_seqs, k,
                                               stride)
        self.k, self.stride, self.mask = k, stride, mask
        if not self._h:
            raise ValueError("invalid k or stride")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_index_free(h)
            self._h = None

    @property
    def n_postings(self) -> int:
        return int(self._lib.or_index_n_postings(self._h))

    def buckets(self):
        """(bucket_start[4^k+1], post_seq[P], post_pos[P]) as numpy copies."""
        nb = (1 << (2 * self.k)) + 1
        P = self.n_postings
        bs = _arr(self._lib.or_index_bucket_start(self._h), nb, np.dtype("<u8"))
        ps = _arr(self._lib.or_index_post_seq(self._h), P, np.dtype("<u4"))
        pp = _arr(self._lib.or_index_post_pos(self._h), P, np.dtype("<u4"))
        return bs, ps, pp

    def search_one(self, query: bytes, params: Params) -> QueryResult:
        q = np.frombuffer(query, dtype=np.uint8)
        r = _Result()
        cp = params._c()
        self._lib.or_search_one(self._h, q.ctypes.data, len(q), ctypes.byref(cp), ctypes.byref(r))
        out = _convert(r)
        self._lib.or_result_free(ctypes.byref(r))
        return out

    def search(self, queries, params: Params, threads: int = 1) -> list[QueryResult]:
        """All queries of a ``synth.Queries`` (or a list of byte strings)."""
        if isinstance(queries, (list, tuple)):
            import synth
            queries = synth.queries_from_strings(queries)
        if params.both_strands:
            import synth
            doubled = []
            for i in range(queries.n):
                q = queries.query(i)
                doubled += [q, reverse_complement(q)]
            queries = synth.queries_from_strings(doubled)
        n = queries.n
        qb = np.ascontiguousarray(queries.bases, dtype=np.uint8)
        qs = np.ascontiguousarray(queries.start, dtype=np.uint64)
        res = (_Result * max(n, 1))()
        cp = params._c()
        self._lib.or_search_batch(self._h, qb.ctypes.data, qs.ctypes.data, n, ctypes.byref(cp), int(threads),
                                  ctypes.cast(res, ctypes.c_void_p))
        out = [_convert(res[i]) for i in range(n)]
        self._lib.or_result_free_batch(ctypes.cast(res, ctypes.c_void_p), n)
        return out


# ---------------------------------------------------------------- pieces --
_COMPLEMENT = bytes.maketrans(b"ACGTUacgtu", b"TGCAAtgcaa")


def reverse_complement(seq) -> bytes:
    """The other strand read 5' to 3': bases reversed, A <-> T and C <-> G (either case),
    U read as T (so it pairs with A); any other byte (a non-base) is kept."""
    return bytes(seq).translate(_COMPLEMENT)[::-1]


def _b(s) -> np.ndarray:
    return np.frombuffer(s.encode() if isinstance(s, str) else bytes(s), dtype=np.uint8)


def extend(query, subject, hsp, params: Params):
    """Phase 3 on one HSP given as (qs, qe, ds, de); returns the extended (qs, qe, ds, de)."""
    lib = _load()
    q, s = _b(query), _b(subject)
    qs, qe, ds, de = hsp
    h = _Hsp(0, qs, qe, ds, de, 0)
    cp = params._c()
    lib.or_extend(q.ctypes.data, len(q), s.ctypes.data, len(s), ctypes.byref(cp), ctypes.byref(h))
    return (h.qs, h.qe, h.ds, h.de)


def banded_sw(query, subject, hsp, params: Params):
    """Phase 6 on one HSP (qs, qe, ds, de); returns (score, qs, qe, ds, de)."""
    lib = _load()
    q, s = _b(query), _b(subject)
    qs, qe, ds, de = hsp
    h = _Hsp(0, qs, qe, ds, de, min(qe - qs, de - ds))
    a = _Aln()
    cp = params._c()
    lib.or_banded_sw(q.ctypes.data, len(q), s.ctypes.data, len(s), ctypes.byref(h), ctypes.byref(cp),
                     ctypes.byref(a))
    return (a.score, a.qs, a.qe, a.ds, a.de)


def merge_overlaps(hsps):
    """Phase 4 on a list of (seq, qs, qe, ds, de); returns the merged boxes in sweep order."""
    lib = _load()
    arr = np.zeros(len(hsps), dtype=HSP_DTYPE)
    for i, (seq, qs, qe, ds, de) in enumerate(hsps):
        arr[i] = (seq, qs, qe, ds, de, min(qe - qs, de - ds))
    out = np.zeros(max(len(hsps), 1), dtype=HSP_DTYPE)
    n = lib.or_merge_overlaps(arr.ctypes.data, len(hsps), out.ctypes.data)
    return [tuple(int(x) for x in r)[:5] for r in out[:n]]


def rank(alns, m: float, n_bank: float, params: Params):
    """Phase 7 on a list of (seq, qs, qe, ds, de, score); returns (seq, qs, qe, ds, de, score, rank)."""
    lib = _load()
    arr = np.zeros(max(len(alns), 1), dtype=ALN_DTYPE)
    for i, (seq, qs, qe, ds, de, sc) in enumerate(alns):
        arr[i]["seq"], arr[i]["qs"], arr[i]["qe"], arr[i]["ds"], arr[i]["de"], arr[i]["score"] = seq, qs, qe, ds, de, sc
    out = np.zeros(max(len(alns), 1), dtype=ALN_DTYPE)
    cp = params._c()
    n = lib.or_rank(arr.ctypes.data, len(alns), float(m), float(n_bank), ctypes.byref(cp), out.ctypes.data)
    return [tuple(int(r[f]) for f in ("seq", "qs", "qe", "ds", "de", "score", "rank")) for r in out[:n]]


def evalue(score: int, m: float, n: float, params: Params) -> float:
    lib = _load()
    cp = params._c()
    return lib.or_evalue(int(score), float(m), float(n), ctypes.byref(cp))


def bits(score: int, params: Params) -> float:
    lib = _load()
    cp = params._c()
    return lib.or_bits(int(score), ctypes.byref(cp))
