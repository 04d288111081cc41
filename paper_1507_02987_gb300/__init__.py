"""Genoogle search path on GB300: Python binding of the C ABI in ``include/genoogle.h``.

This module only marshals arguments: every phase of the search runs in the
CUDA library ``_build/libgenoogle.so`` (built by ``_build.build()``).  Importing
works without a GPU; any call that needs the device fails with a CUDA error
when none is present, and loading fails loudly when the library is missing.

The functions ``gn_*`` mirror the C entry points one to one.  ``Index`` and
``search`` are conveniences over them that accept numpy arrays (host memory) or
torch tensors (host or CUDA memory) and return numpy structured arrays.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import _build

__all__ = ["GnError", "load", "Index", "search", "HIT_DTYPE", "HSP_DTYPE"]

GN_OK, GN_EINVAL, GN_ENOMEM, GN_ECUDA, GN_ETIMEOUT, GN_EBUSY, GN_ETOOBIG, GN_EINTERNAL = range(8)
GN_MEM_HOST, GN_MEM_DEVICE = 0, 1
GN_FLAG_KEEP_STAGES, GN_FLAG_KEEP_HITS, GN_FLAG_TIME_KERNELS, GN_FLAG_BOTH_STRANDS = 1, 2, 4, 8
GN_TUNE_BAND, GN_TUNE_KERNELS = 1, 2
GN_STAGE_HSP, GN_STAGE_EXT, GN_STAGE_MERGED, GN_STAGE_SELECTED, GN_STAGE_ALIGNED, GN_STAGE_HITS, \
    GN_STAGE_HIT_COUNTS = range(7)
STATUS_NAMES = {0: "GN_OK", 1: "GN_EINVAL", 2: "GN_ENOMEM", 3: "GN_ECUDA", 4: "GN_ETIMEOUT", 5: "GN_EBUSY",
                6: "GN_ETOOBIG", 7: "GN_EINTERNAL"}


class GnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gn_bank(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_uint32), ("seq_start", ctypes.c_void_p), ("bases", ctypes.c_void_p),
                ("bases_mem", ctypes.c_int)]


class gn_queries(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("start", ctypes.c_void_p), ("bases", ctypes.c_void_p),
                ("bases_mem", ctypes.c_int)]


class gn_scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("lambda_", ctypes.c_double), ("K", ctypes.c_double)]


class gn_params(ctypes.Structure):
    _fields_ = [("max_hit_distance", ctypes.c_uint32), ("min_hsp_len", ctypes.c_uint32),
                ("xdrop", ctypes.c_int32), ("max_alignments", ctypes.c_uint32), ("band_w", ctypes.c_uint32),
                ("max_evalue", ctypes.c_double), ("flags", ctypes.c_uint32)]


class gn_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("tile_hits", "fill_threads", "bucket_target", "sw_lanes",
                                                "sw_wave_rows", "reserved")]


class gn_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("requests", "batches", "max_batch", "max_concurrent",
                                                 "peak_in_use", "in_use", "queued")]


class gn_int_peaks(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("add3_ops", "addmax_plain_ops", "dpx_addmax_ops", "dpx_max3_ops",
                                                "dpx_bmax_ops")] + [("sms", ctypes.c_uint32)]


class gn_index_info(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("stride", ctypes.c_int32), ("n_seqs", ctypes.c_uint32),
                ("n_bases", ctypes.c_uint64), ("n_postings", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64)]


HIT_DTYPE = np.dtype([("query", "<u4"), ("seq", "<u4"), ("q_start", "<u4"), ("q_end", "<u4"),
                      ("db_start", "<u4"), ("db_end", "<u4"), ("score", "<i4"), ("rank", "<u4"),
                      ("evalue", "<f8"), ("bits", "<f8")])
HSP_DTYPE = np.dtype([("query", "<u4"), ("seq", "<u4"), ("q_start", "<u4"), ("q_end", "<u4"),
                      ("db_start", "<u4"), ("db_end", "<u4"), ("len", "<u4")])
STAGE_HIT_DTYPE = np.dtype([("query", "<u4"), ("qpos", "<u4"), ("seq", "<u4"), ("pos", "<u4")])

_lib = None
_lock = threading.Lock()


def load():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # GN_LIBRARY=checks selects the checked build (device-side bounds checks) of the same library
        path = _build.CHECKS_LIB if os.environ.get("GN_LIBRARY") == "checks" else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1507_02987_gb300._build.build() "
                              "(the search runs only in the CUDA library; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
        st = ctypes.c_int
        sig = {
            "gn_default_params": (st, [ctypes.POINTER(gn_scoring), ctypes.POINTER(gn_params)]),
            "gn_index_build": (st, [ctypes.POINTER(gn_bank), ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]),
            "gn_index_free": (None, [vp]),
            "gn_index_get_info": (st, [vp, ctypes.POINTER(gn_index_info)]),
            "gn_index_export": (st, [vp, vp, vp, vp]),
            "gn_search": (st, [vp, ctypes.POINTER(gn_queries), ctypes.POINTER(gn_scoring), ctypes.POINTER(gn_params),
                               vp, ctypes.POINTER(vp)]),
            "gn_results_free": (None, [vp]),
            "gn_results_get": (st, [vp, u32, ctypes.POINTER(vp), ctypes.POINTER(u32)]),
            "gn_results_count": (st, [vp, ctypes.POINTER(u32), ctypes.POINTER(u64)]),
            "gn_results_stage": (st, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(u64)]),
            "gn_last_phase_times": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_char_p),
                                                   ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
            "gn_last_kernel_times": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_char_p),
                                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32),
                                                    ctypes.POINTER(u64), ctypes.c_int]),
            "gn_kernel_launch_count": (u64, []),
            "gn_index_build_masked": (st, [ctypes.POINTER(gn_bank), ctypes.c_char_p, ctypes.c_int, vp,
                                           ctypes.POINTER(vp)]),
            "gn_index_save": (st, [vp, ctypes.c_char_p]),
            "gn_index_set_tuning": (st, [vp, ctypes.POINTER(gn_tuning)]),
            "gn_index_get_tuning": (st, [vp, ctypes.POINTER(gn_tuning)]),
            "gn_autotune": (st, [vp, ctypes.POINTER(gn_queries), ctypes.POINTER(gn_scoring), ctypes.POINTER(gn_params),
                                 u32, vp, ctypes.POINTER(gn_tuning)]),
            "gn_index_load": (st, [ctypes.c_char_p, ctypes.POINTER(vp)]),
            "gn_serve_start": (st, [vp, ctypes.POINTER(gn_scoring), ctypes.POINTER(gn_params), u64,
                                    ctypes.POINTER(vp)]),
            "gn_serve_submit": (st, [vp, ctypes.c_char_p, u32, ctypes.POINTER(u64)]),
            "gn_serve_poll": (st, [vp, u64, u32, ctypes.POINTER(vp)]),
            "gn_serve_poll_any": (st, [vp, u32, ctypes.POINTER(u64), ctypes.POINTER(vp)]),
            "gn_serve_get_stats": (st, [vp, ctypes.POINTER(gn_serve_stats)]),
            "gn_serve_stop": (st, [vp]),
            "gn_align_hsps_static": (st, [vp, vp, vp, u32, vp, u32, ctypes.POINTER(gn_scoring), u32, vp, vp]),
            "gn_measure_int_peaks": (st, [ctypes.POINTER(gn_int_peaks), vp]),
            "gn_debug_fail_alloc": (None, [u64]),
            "gn_debug_scan": (st, [vp, vp, u64, u64, ctypes.c_int, vp]),
            "gn_debug_sort": (st, [vp, vp, u64, ctypes.c_int, ctypes.c_int, u64, ctypes.c_int, ctypes.c_int, vp]),
            "gn_debug_alloc_count": (u64, []),
            "gn_debug_live_allocs": (ctypes.c_int64, []),
            "gn_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(status: int):
    if status != GN_OK:
        raise GnError(status, load().gn_last_error().decode(errors="replace"))


# ------------------------------------------------------------ raw ABI --
def gn_measure_int_peaks(stream: int = 0) -> dict:
    """Measured integer-pipe throughput of the current GPU (operations per second)."""
    o = gn_int_peaks()
    _check(load().gn_measure_int_peaks(ctypes.byref(o), ctypes.c_void_p(stream)))
    return {n: getattr(o, n) for n, _ in gn_int_peaks._fields_}


def gn_debug_fail_alloc(nth: int):
    """The nth device allocation of a search from now on fails (GN_ENOMEM); 0 disables."""
    load().gn_debug_fail_alloc(nth)


def gn_debug_scan(in_ptr: int, out_ptr: int, n: int, wait_cycles: int = 0, drop_first: bool = False,
                  stream: int = 0):
    """The library's single-pass scan on device buffers (tests of its bounded wait)."""
    _check(load().gn_debug_scan(ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), n, wait_cycles,
                                1 if drop_first else 0, ctypes.c_void_p(stream)))


def gn_debug_sort(keys_ptr: int, vals_ptr: int | None, n: int, bit_lo: int, bit_hi: int, wait_cycles: int = 0,
                  drop_first: bool = False, three_kernel: bool = False, stream: int = 0):
    """The library's radix sort on device buffers, in place (tests of both forms and of the
    single-pass form's bounded wait)."""
    _check(load().gn_debug_sort(ctypes.c_void_p(keys_ptr), ctypes.c_void_p(vals_ptr or 0), n, bit_lo, bit_hi,
                                wait_cycles, 1 if drop_first else 0, 1 if three_kernel else 0,
                                ctypes.c_void_p(stream)))


def gn_debug_alloc_count() -> int:
    return int(load().gn_debug_alloc_count())


def gn_debug_live_allocs() -> int:
    return int(load().gn_debug_live_allocs())


def gn_default_params():
    sc, p = gn_scoring(), gn_params()
    _check(load().gn_default_params(ctypes.byref(sc), ctypes.byref(p)))
    return sc, p


def gn_index_build(bank: gn_bank, k: int, stride: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().gn_index_build(ctypes.byref(bank), k, stride, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h.value


def gn_index_build_masked(bank: gn_bank, mask: str, stride: int, stream: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load().gn_index_build_masked(ctypes.byref(bank), mask.encode(), stride, ctypes.c_void_p(stream),
                                        ctypes.byref(h)))
    return h.value


def gn_index_save(h: int, path: str):
    _check(load().gn_index_save(ctypes.c_void_p(h), os.fsencode(path)))


def gn_index_load(path: str) -> int:
    r = ctypes.c_void_p()
    _check(load().gn_index_load(os.fsencode(path), ctypes.byref(r)))
    return r.value


def gn_index_free(h: int):
    load().gn_index_free(ctypes.c_void_p(h))


def gn_index_get_info(h: int) -> gn_index_info:
    info = gn_index_info()
    _check(load().gn_index_get_info(ctypes.c_void_p(h), ctypes.byref(info)))
    return info


def gn_index_export(h: int, bucket_start=None, post_seq=None, post_pos=None):
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)
    _check(load().gn_index_export(ctypes.c_void_p(h), ptr(bucket_start), ptr(post_seq), ptr(post_pos)))


def gn_search(h: int, queries: gn_queries, scoring: gn_scoring, params: gn_params, stream: int = 0) -> int:
    r = ctypes.c_void_p()
    _check(load().gn_search(ctypes.c_void_p(h), ctypes.byref(queries), ctypes.byref(scoring),
                            ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(r)))
    return r.value


def gn_results_free(r: int):
    load().gn_results_free(ctypes.c_void_p(r))


def gn_results_get(r: int, query: int) -> np.ndarray:
    p, n = ctypes.c_void_p(), ctypes.c_uint32()
    _check(load().gn_results_get(ctypes.c_void_p(r), query, ctypes.byref(p), ctypes.byref(n)))
    return _copy(p.value, n.value, HIT_DTYPE)


def gn_results_count(r: int):
    nq, nh = ctypes.c_uint32(), ctypes.c_uint64()
    _check(load().gn_results_count(ctypes.c_void_p(r), ctypes.byref(nq), ctypes.byref(nh)))
    return nq.value, nh.value


_STAGE_DTYPES = {GN_STAGE_HSP: HSP_DTYPE, GN_STAGE_EXT: HSP_DTYPE, GN_STAGE_MERGED: HSP_DTYPE,
                 GN_STAGE_SELECTED: HSP_DTYPE, GN_STAGE_ALIGNED: HIT_DTYPE, GN_STAGE_HITS: STAGE_HIT_DTYPE,
                 GN_STAGE_HIT_COUNTS: np.dtype("<u8")}


def gn_results_stage(r: int, stage: int) -> np.ndarray:
    p, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(load().gn_results_stage(ctypes.c_void_p(r), stage, ctypes.byref(p), ctypes.byref(n)))
    return _copy(p.value, n.value, _STAGE_DTYPES[stage])


def gn_last_phase_times(h: int) -> dict:
    names = (ctypes.c_char_p * 64)()
    ms = (ctypes.c_float * 64)()
    n = load().gn_last_phase_times(ctypes.c_void_p(h), names, ms, 64)
    out = {}
    for i in range(n):
        key = names[i].decode()
        out[key] = out.get(key, 0.0) + ms[i]
    return out


def gn_last_kernel_times(h: int) -> dict:
    """{kernel name: (total ms, launches, work items)} of the last search run with GN_FLAG_TIME_KERNELS."""
    names = (ctypes.c_char_p * 128)()
    ms = (ctypes.c_double * 128)()
    la = (ctypes.c_uint32 * 128)()
    un = (ctypes.c_uint64 * 128)()
    n = load().gn_last_kernel_times(ctypes.c_void_p(h), names, ms, la, un, 128)
    return {names[i].decode(): (ms[i], la[i], un[i]) for i in range(n)}


def gn_kernel_launch_count() -> int:
    return int(load().gn_kernel_launch_count())


def gn_serve_start(h: int, scoring: gn_scoring, params: gn_params, mem_budget: int) -> int:
    s = ctypes.c_void_p()
    _check(load().gn_serve_start(ctypes.c_void_p(h), ctypes.byref(scoring), ctypes.byref(params), mem_budget,
                                 ctypes.byref(s)))
    return s.value


def gn_serve_submit(s: int, bases: bytes) -> int:
    t = ctypes.c_uint64()
    _check(load().gn_serve_submit(ctypes.c_void_p(s), bases, len(bases), ctypes.byref(t)))
    return t.value


def gn_serve_poll(s: int, ticket: int, timeout_ms: int):
    """Returns a results handle, or None on GN_ETIMEOUT."""
    r = ctypes.c_void_p()
    st = load().gn_serve_poll(ctypes.c_void_p(s), ticket, timeout_ms, ctypes.byref(r))
    if st == GN_ETIMEOUT:
        return None
    _check(st)
    return r.value


def gn_serve_poll_any(s: int, timeout_ms: int):
    """(ticket, results handle) of the oldest finished request, or None on GN_ETIMEOUT.
    A failed request raises GnError."""
    r = ctypes.c_void_p()
    t = ctypes.c_uint64()
    st = load().gn_serve_poll_any(ctypes.c_void_p(s), timeout_ms, ctypes.byref(t), ctypes.byref(r))
    if st == GN_ETIMEOUT:
        return None
    _check(st)
    return t.value, r.value


def gn_serve_get_stats(s: int) -> dict:
    o = gn_serve_stats()
    _check(load().gn_serve_get_stats(ctypes.c_void_p(s), ctypes.byref(o)))
    return {n: int(getattr(o, n)) for n, _ in gn_serve_stats._fields_}


def gn_serve_stop(s: int):
    _check(load().gn_serve_stop(ctypes.c_void_p(s)))


def gn_align_hsps_static(h: int, query_bases_dev: int, query_start_dev: int, n_queries: int, hsps_dev: int,
                         n_hsps: int, scoring: gn_scoring, band_w: int, out_dev: int, stream: int = 0):
    """Allocation-free alignment of caller-given HSPs; every pointer is a device address."""
    _check(load().gn_align_hsps_static(ctypes.c_void_p(h), ctypes.c_void_p(query_bases_dev),
                                       ctypes.c_void_p(query_start_dev), n_queries, ctypes.c_void_p(hsps_dev),
                                       n_hsps, ctypes.byref(scoring), band_w, ctypes.c_void_p(out_dev),
                                       ctypes.c_void_p(stream)))


def gn_last_error() -> str:
    return load().gn_last_error().decode(errors="replace")


def _copy(ptr, n, dtype):
    if not n or not ptr:
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (n * dtype.itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype).copy()


# -------------------------------------------------------- conveniences --
def _buffer(x):
    """(pointer, memory kind, keepalive) of a numpy array or a torch tensor (host or CUDA)."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x)
        return x.ctypes.data, GN_MEM_HOST, x
    if isinstance(x, (bytes, bytearray)):
        a = np.frombuffer(bytes(x), dtype=np.uint8)
        return a.ctypes.data, GN_MEM_HOST, a
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        x = x.contiguous()
        return x.data_ptr(), (GN_MEM_DEVICE if x.is_cuda else GN_MEM_HOST), x
    raise TypeError(f"unsupported buffer type {type(x)}")


def make_scoring(match=1, mismatch=-3, gap_open=-5, gap_extend=-2, lam=1.3740631, K=0.711) -> gn_scoring:
    return gn_scoring(match, mismatch, gap_open, gap_extend, lam, K)


def make_params(max_hit_distance=0, min_hsp_len=0, xdrop=20, max_alignments=100, band_w=16,
                max_evalue=math.inf, flags=0) -> gn_params:
    return gn_params(max_hit_distance, min_hsp_len, xdrop, max_alignments, band_w, max_evalue, flags)


class Index:
    """A device-resident index of a bank (sequences back to back + starts)."""

    def __init__(self, seq_start, bases, k: int = 11, stride: int = 11, stream: int = 0, mask: str | None = None):
        """k-mer windows, or with ``mask`` (e.g. "111010010100110111") spaced seeds of the mask's
        length keyed by their kept bases; k is then the mask's number of ones."""
        ss = np.ascontiguousarray(seq_start, dtype=np.uint64)
        ptr, mem, keep = _buffer(bases)
        self._keep = (ss, keep)
        bank = gn_bank(len(ss) - 1, ss.ctypes.data, ptr, mem)
        if mask is not None:
            self.handle = gn_index_build_masked(bank, mask, stride, stream)
            k = mask.count("1")
        else:
            self.handle = gn_index_build(bank, k, stride, stream)
        self._keep = None
        self.k, self.stride, self.mask = k, stride, mask

    @classmethod
    def from_bank(cls, bank, k=11, stride=11, stream=0, mask=None):
        return cls(bank.seq_start, bank.bases, k, stride, stream, mask)

    @classmethod
    def load(cls, path: str) -> "Index":
        """An index read back from a file written by save()."""
        self = cls.__new__(cls)
        self._keep = None
        self.handle = gn_index_load(path)
        info = gn_index_get_info(self.handle)
        self.k, self.stride, self.mask = info.k, info.stride, None
        return self

    def save(self, path: str):
        gn_index_save(self.handle, path)

    def info(self) -> gn_index_info:
        return gn_index_get_info(self.handle)

    def export(self):
        info = self.info()
        bs = np.zeros((1 << (2 * self.k)) + 1, dtype=np.uint64)
        ps = np.zeros(info.n_postings, dtype=np.uint32)
        pp = np.zeros(info.n_postings, dtype=np.uint32)
        gn_index_export(self.handle, bs, ps, pp)
        return bs, ps, pp

    def phase_times(self) -> dict:
        return gn_last_phase_times(self.handle)

    def kernel_times(self) -> dict:
        return gn_last_kernel_times(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            gn_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Results:
    """Owns a gn_results handle."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def n_queries(self) -> int:
        return gn_results_count(self.handle)[0]

    def query(self, i: int) -> np.ndarray:
        return gn_results_get(self.handle, i)

    def all(self) -> list[np.ndarray]:
        return [self.query(i) for i in range(self.n_queries)]

    def stage(self, stage: int) -> np.ndarray:
        return gn_results_stage(self.handle, stage)

    def close(self):
        if getattr(self, "handle", None):
            gn_results_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A request loop over a resident index (gn_serve_*); results are Results of one query."""

    def __init__(self, index: Index, mem_budget: int, scoring: gn_scoring | None = None,
                 params: gn_params | None = None):
        self.index = index  # keeps the index alive while the server runs
        sc = scoring if scoring is not None else make_scoring()
        p = params if params is not None else make_params()
        self.handle = gn_serve_start(index.handle, sc, p, mem_budget)

    def submit(self, bases) -> int:
        return gn_serve_submit(self.handle, bytes(bases))

    def poll(self, ticket: int, timeout_ms: int = 60000):
        h = gn_serve_poll(self.handle, ticket, timeout_ms)
        return None if h is None else Results(h)

    def poll_any(self, timeout_ms: int = 60000):
        got = gn_serve_poll_any(self.handle, timeout_ms)
        return None if got is None else (got[0], Results(got[1]))

    def stats(self) -> dict:
        return gn_serve_get_stats(self.handle)

    def stop(self):
        if getattr(self, "handle", None):
            gn_serve_stop(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def set_tuning(index: Index, tile_hits=0, fill_threads=0, bucket_target=0, sw_lanes=0, sw_wave_rows=0):
    _check(load().gn_index_set_tuning(ctypes.c_void_p(index.handle),
                                      ctypes.byref(gn_tuning(tile_hits, fill_threads, bucket_target, sw_lanes,
                                                             sw_wave_rows, 0))))


def get_tuning(index: Index) -> dict:
    t = gn_tuning()
    _check(load().gn_index_get_tuning(ctypes.c_void_p(index.handle), ctypes.byref(t)))
    return {n: int(getattr(t, n)) for n, _ in gn_tuning._fields_ if n != "reserved"}


def autotune(index: Index, start, bases, scoring: gn_scoring | None = None, params: gn_params | None = None,
             what: int = GN_TUNE_BAND | GN_TUNE_KERNELS, stream: int = 0):
    """Runs the autotuner on a calibration sample; returns (params with the chosen band_w, tuning dict).
    The kernel tuning is installed on the index."""
    st = np.ascontiguousarray(start, dtype=np.uint64)
    ptr, mem, keep = _buffer(bases)
    q = gn_queries(len(st) - 1, st.ctypes.data, ptr, mem)
    sc = scoring if scoring is not None else make_scoring()
    p = params if params is not None else make_params()
    p = gn_params.from_buffer_copy(p)
    t = gn_tuning()
    _check(load().gn_autotune(ctypes.c_void_p(index.handle), ctypes.byref(q), ctypes.byref(sc), ctypes.byref(p),
                              what, ctypes.c_void_p(stream), ctypes.byref(t)))
    del keep
    return p, {n: int(getattr(t, n)) for n, _ in gn_tuning._fields_ if n != "reserved"}


def search(index: Index, start, bases, scoring: gn_scoring | None = None, params: gn_params | None = None,
           stream: int = 0) -> Results:
    """Searches queries (bases[start[i]:start[i+1]]); bases may be host or device memory."""
    st = np.ascontiguousarray(start, dtype=np.uint64)
    ptr, mem, keep = _buffer(bases)
    q = gn_queries(len(st) - 1, st.ctypes.data, ptr, mem)
    sc = scoring if scoring is not None else make_scoring()
    p = params if params is not None else make_params()
    h = gn_search(index.handle, q, sc, p, stream)
    del keep
    return Results(h)
