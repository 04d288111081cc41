"""Seeded synthetic workloads shaped like the paper's experiments (Results section).

The paper searches hs_phase3 + RefSeq (4.25 Gbp) with query sets of one bank
sequence plus mutated copies.  Those data are not available; this module
generates stand-ins from a seed.  It holds none of the method's arithmetic and is
the only code shared by the CUDA-path tests, the oracle tests and the benchmark.

Recipes (one per workload; base seed 0x6E000000 + workload index):

* tiny     - 1,000 sequences, lengths U[500, 2000], uniform ACGT; 10 queries of
             length U[300, 1000] copied from random bank substrings with 5 %
             substitutions and 1 % single-base indels.
* mid      - 200,000 sequences, log-normal lengths (median 1,500, sigma 0.7585,
             clipped to [100, 50,000]; ~400 Mbp), per-sequence GC ~ U[0.35, 0.65],
             500 repeat families (consensus length log-uniform 300-6,000) whose
             copies (1-10 % divergence) overwrite 20 % of the bases; 1,000
             queries, log-uniform 80-10,000 bp, planted homologs at 2-25 %
             divergence (substitution:indel = 5:1).
* batched  - the mid bank; 10,000 queries, log-uniform 50-5,000 bp, half planted
             homologs at 0-30 % divergence, half uniform random.
* large    - 2.5 M sequences, log-normal lengths (median 1,200, same sigma,
             clipped to [100, 200,000]; ~4 Gbp), GC and repeats as mid; 2,000
             queries, log-uniform 200-20,000 bp, half planted homologs at 2-25 %.
* serving  - the large bank; requests log-uniform 50-20,000 bp, 30 % homologs,
             open-loop Poisson arrivals.
* long     - the large bank; 40 queries log-uniform 65,536 bp - 1 Mbp (the size
             range of the paper's longest query sets), half planted homologs at
             2-25 % divergence (a homolog is at most as long as the longest bank
             sequence, 200,000 bp).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgn_synth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 0x6E000000
WORKLOADS = ("tiny", "mid", "batched", "large", "serving")


def build(force: bool = False) -> str:
    """Compile the generator (plain C, no architecture-specific flags)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _BankSpec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_seqs", ctypes.c_uint32), ("len_dist", ctypes.c_int32),
                ("len_median", ctypes.c_double), ("len_sigma", ctypes.c_double),
                ("len_lo", ctypes.c_uint32), ("len_hi", ctypes.c_uint32),
                ("gc_lo", ctypes.c_double), ("gc_hi", ctypes.c_double),
                ("n_families", ctypes.c_uint32), ("fam_len_lo", ctypes.c_uint32),
                ("fam_len_hi", ctypes.c_uint32), ("fam_div_lo", ctypes.c_double),
                ("fam_div_hi", ctypes.c_double), ("repeat_frac", ctypes.c_double),
                ("n_threads", ctypes.c_int32)]


class _QuerySpec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_queries", ctypes.c_uint32), ("len_dist", ctypes.c_int32),
                ("len_lo", ctypes.c_uint32), ("len_hi", ctypes.c_uint32),
                ("homolog_frac", ctypes.c_double), ("div_lo", ctypes.c_double), ("div_hi", ctypes.c_double),
                ("p_sub", ctypes.c_double), ("p_indel", ctypes.c_double), ("random_gc", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.synth_bank_layout.restype = ctypes.c_uint64
            lib.synth_bank_layout.argtypes = [ctypes.POINTER(_BankSpec), u64p]
            lib.synth_bank_fill.restype = None
            lib.synth_bank_fill.argtypes = [ctypes.POINTER(_BankSpec), u64p, ctypes.c_void_p]
            lib.synth_queries_plan.restype = ctypes.c_uint64
            lib.synth_queries_plan.argtypes = [ctypes.POINTER(_QuerySpec), u64p, ctypes.c_uint32, u64p]
            lib.synth_queries_fill.restype = ctypes.c_uint64
            lib.synth_queries_fill.argtypes = [ctypes.POINTER(_QuerySpec), u64p, u64p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_uint64, u64p]
            lib.synth_poisson_arrivals.restype = None
            lib.synth_poisson_arrivals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                                   ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class BankSpec:
    seed: int
    n_seqs: int
    len_dist: int           # 0 uniform, 1 log-normal
    len_median: float
    len_sigma: float
    len_lo: int
    len_hi: int
    gc_lo: float = 0.5
    gc_hi: float = 0.5
    n_families: int = 0
    fam_len_lo: int = 300
    fam_len_hi: int = 6000
    fam_div_lo: float = 0.01
    fam_div_hi: float = 0.10
    repeat_frac: float = 0.0


@dataclass(frozen=True)
class QuerySpec:
    seed: int
    n_queries: int
    len_dist: int           # 0 uniform, 1 log-uniform
    len_lo: int
    len_hi: int
    homolog_frac: float
    div_lo: float = 0.0
    div_hi: float = 0.0
    p_sub: float = -1.0     # >= 0: fixed per-base rates instead of the divergence model
    p_indel: float = 0.0
    random_gc: float = 0.5


_SIGMA = 0.7585  # log-normal sigma giving mean ~ 1.33 x median

BANKS = {
    "tiny": BankSpec(BASE_SEED + 0, 1000, 0, 0.0, 0.0, 500, 2000),
    "mid": BankSpec(BASE_SEED + 1, 200_000, 1, 1500.0, _SIGMA, 100, 50_000, 0.35, 0.65, 500, 300, 6000,
                    0.01, 0.10, 0.20),
    "large": BankSpec(BASE_SEED + 3, 2_500_000, 1, 1200.0, _SIGMA, 100, 200_000, 0.35, 0.65, 500, 300, 6000,
                      0.01, 0.10, 0.20),
}
BANK_OF = {"tiny": "tiny", "mid": "mid", "batched": "mid", "large": "large", "serving": "large", "long": "large"}

QUERIES = {
    "tiny": QuerySpec(BASE_SEED + 0, 10, 0, 300, 1000, 1.0, p_sub=0.05, p_indel=0.01),
    "mid": QuerySpec(BASE_SEED + 1, 1000, 1, 80, 10_000, 1.0, 0.02, 0.25),
    "batched": QuerySpec(BASE_SEED + 2, 10_000, 1, 50, 5_000, 0.5, 0.0, 0.30),
    "large": QuerySpec(BASE_SEED + 3, 2000, 1, 200, 20_000, 0.5, 0.02, 0.25),
    "serving": QuerySpec(BASE_SEED + 4, 4000, 1, 50, 20_000, 0.3, 0.02, 0.25),
    "long": QuerySpec(BASE_SEED + 5, 40, 1, 65_536, 1_000_000, 0.5, 0.02, 0.25),
}


@dataclass
class Bank:
    """Sequences back to back: sequence s is bases[seq_start[s]:seq_start[s+1]] (ASCII)."""
    seq_start: np.ndarray   # uint64, n_seqs + 1
    bases: np.ndarray       # uint8 ASCII
    spec: BankSpec

    @property
    def n_seqs(self) -> int:
        return len(self.seq_start) - 1

    @property
    def n_bases(self) -> int:
        return int(self.seq_start[-1])

    def seq(self, s: int) -> bytes:
        return self.bases[int(self.seq_start[s]):int(self.seq_start[s + 1])].tobytes()


@dataclass
class Queries:
    start: np.ndarray       # uint64, n + 1
    bases: np.ndarray       # uint8 ASCII
    meta: np.ndarray        # uint64 [n, 5]: is_homolog, src_seq, src_pos, src_len, divergence*1e6
    spec: QuerySpec

    @property
    def n(self) -> int:
        return len(self.start) - 1

    def query(self, i: int) -> bytes:
        return self.bases[int(self.start[i]):int(self.start[i + 1])].tobytes()

    def subset(self, idx) -> "Queries":
        idx = list(idx)
        parts = [self.bases[int(self.start[i]):int(self.start[i + 1])] for i in idx]
        lens = np.array([len(p) for p in parts], dtype=np.uint64)
        start = np.zeros(len(idx) + 1, dtype=np.uint64)
        start[1:] = np.cumsum(lens)
        bases = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
        return Queries(start, bases.astype(np.uint8), self.meta[idx], self.spec)


def _u64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def make_bank(spec: BankSpec | str, n_seqs: int | None = None, threads: int | None = None,
              alloc=None) -> Bank:
    """Generate a bank.  ``alloc(nbytes) -> (numpy uint8 array)`` may supply the base buffer
    (e.g. pinned host memory); the bases are identical whatever buffer is used."""
    if isinstance(spec, str):
        spec = BANKS[BANK_OF[spec]]
    if n_seqs is not None:
        spec = replace(spec, n_seqs=int(n_seqs))
    lib = _load()
    cs = _BankSpec(spec.seed, spec.n_seqs, spec.len_dist, spec.len_median, spec.len_sigma, spec.len_lo,
                   spec.len_hi, spec.gc_lo, spec.gc_hi, spec.n_families, spec.fam_len_lo, spec.fam_len_hi,
                   spec.fam_div_lo, spec.fam_div_hi, spec.repeat_frac,
                   int(threads or min(16, os.cpu_count() or 1)))
    seq_start = np.zeros(spec.n_seqs + 1, dtype=np.uint64)
    total = lib.synth_bank_layout(ctypes.byref(cs), _u64p(seq_start))
    bases = alloc(total) if alloc is not None else np.empty(total, dtype=np.uint8)
    lib.synth_bank_fill(ctypes.byref(cs), _u64p(seq_start), ctypes.c_void_p(bases.ctypes.data))
    return Bank(seq_start, bases, spec)


def make_queries(spec: QuerySpec | str, bank: Bank, n: int | None = None) -> Queries:
    if isinstance(spec, str):
        spec = QUERIES[spec]
    if n is not None:
        spec = replace(spec, n_queries=int(n))
    lib = _load()
    cs = _QuerySpec(spec.seed, spec.n_queries, spec.len_dist, spec.len_lo, spec.len_hi, spec.homolog_frac,
                    spec.div_lo, spec.div_hi, spec.p_sub, spec.p_indel, spec.random_gc)
    meta = np.zeros((spec.n_queries, 5), dtype=np.uint64)
    cap = lib.synth_queries_plan(ctypes.byref(cs), _u64p(bank.seq_start), bank.n_seqs, _u64p(meta))
    out = np.empty(max(cap, 1), dtype=np.uint8)
    start = np.zeros(spec.n_queries + 1, dtype=np.uint64)
    total = lib.synth_queries_fill(ctypes.byref(cs), _u64p(meta), _u64p(bank.seq_start),
                                   ctypes.c_void_p(bank.bases.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                                   cap, _u64p(start))
    return Queries(start, out[:total].copy(), meta, spec)


def poisson_arrivals(rate: float, n: int, seed: int = BASE_SEED + 4) -> np.ndarray:
    """Cumulative arrival times (seconds) of an open-loop Poisson process."""
    lib = _load()
    t = np.zeros(n, dtype=np.float64)
    lib.synth_poisson_arrivals(seed, n, float(rate), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return t


def bank_from_strings(seqs) -> Bank:
    """A bank from explicit sequences (hand-made test cases)."""
    seqs = [s.encode() if isinstance(s, str) else bytes(s) for s in seqs]
    start = np.zeros(len(seqs) + 1, dtype=np.uint64)
    start[1:] = np.cumsum([len(s) for s in seqs]) if seqs else []
    bases = np.frombuffer(b"".join(seqs), dtype=np.uint8).copy()
    return Bank(start, bases, BANKS["tiny"])


def queries_from_strings(qs) -> Queries:
    qs = [s.encode() if isinstance(s, str) else bytes(s) for s in qs]
    start = np.zeros(len(qs) + 1, dtype=np.uint64)
    start[1:] = np.cumsum([len(s) for s in qs]) if qs else []
    bases = np.frombuffer(b"".join(qs), dtype=np.uint8).copy()
    return Queries(start, bases, np.zeros((len(qs), 5), dtype=np.uint64), QUERIES["tiny"])
