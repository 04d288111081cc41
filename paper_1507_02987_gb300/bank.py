"""The formatted data bank on disk.

The paper ("Inverted Indexes") formats a data bank once: every sequence is coded
with 2 bits per base and stored in a disk file together with its name,
identification code and description. At start-up only the metadata (file
offsets among it) is read into memory; a sequence is read from the file when its
information is needed. This module is that storage layer, on the host:

* ``read_fasta`` parses FASTA text into (name, description, sequence) records;
* ``write_bank`` formats records (or a FASTA file) into a bank file;
* ``BankFile`` maps a bank file, holds its metadata and decodes sequences on
  demand (``seq``), or the whole bank (``arrays``) for ``Index``.

Bases A, C, G, T and U in either case take 2 bits (U is coded as T). Every other
byte is a non-base, which the search treats alike (it breaks a seed and scores as a
mismatch), so the file keeps the positions of non-bases as runs and decodes them
as ``N``; case is not kept, as the search ignores it. A search over the decoded
bank therefore gives the same results as over the original text. The
identification code of a sequence is its index in the file, which is the
sequence id of search results.

File layout (little-endian):

====================  =====================================================
header (80 bytes)     magic ``GNOGBNK1``, version, n_seqs, n_bases, n_runs,
                      and the byte offsets of the sections below
seq_start             (n_seqs + 1) x uint64: sequence s is bases
                      [seq_start[s], seq_start[s + 1])
codes                 ceil(n_bases / 4) bytes, 4 bases per byte, the first
                      base in the high bits (A=0, C=1, G=2, T=3)
runs                  n_runs x (uint64 start, uint64 length): non-bases,
                      sorted, disjoint, not adjacent
meta_start            (n_seqs + 1) x uint64 offsets into the metadata blob
meta                  per sequence: name, a 0 byte, description (UTF-8)
====================  =====================================================
"""
from __future__ import annotations

import os
import struct
from dataclasses import dataclass

import numpy as np

MAGIC = b"GNOGBNK1"
VERSION = 1
_HEADER = struct.Struct("<8sIIQQQQQQQQ")  # magic, version, pad, n_seqs, n_bases, n_runs, 5 section offsets
assert _HEADER.size == 80

# byte -> 2-bit code, or 4 for a non-base
_CODE = np.full(256, 4, dtype=np.uint8)
for _c, _v in zip(b"ACGTUacgtu", (0, 1, 2, 3, 3, 0, 1, 2, 3, 3)):
    _CODE[_c] = _v
_LETTER = np.frombuffer(b"ACGTN", dtype=np.uint8)


@dataclass
class Record:
    name: str
    description: str
    sequence: bytes


def read_fasta(source):
    """Yields the records of FASTA text: a path, or an iterable of lines (str or bytes).

    A header line starts with ``>``; its first word is the name and the rest the
    description. Sequence lines are joined with all whitespace removed. Blank lines
    and lines starting with ``;`` are skipped. Sequence text before the first header
    is an error (ValueError)."""
    if isinstance(source, (str, os.PathLike)):
        with open(source, "rb") as f:
            yield from _read_fasta_bytes(f.read())
        return
    name = desc = None
    parts: list[bytes] = []
    for raw in source:
        line = raw.encode() if isinstance(raw, str) else bytes(raw)
        line = line.rstrip(b"\r\n")
        if not line.strip() or line.startswith(b";"):
            continue
        if line.startswith(b">"):
            if name is not None:
                yield Record(name, desc, b"".join(parts))
            head = line[1:].strip().split(None, 1)
            name = head[0].decode("utf-8", "replace") if head else ""
            desc = head[1].decode("utf-8", "replace") if len(head) > 1 else ""
            parts = []
            continue
        if name is None:
            raise ValueError("FASTA sequence text before the first header")
        parts.append(b"".join(line.split()))
    if name is not None:
        yield Record(name, desc, b"".join(parts))


_WS = b" \t\r\n\v\f"


def _line_spans(data: bytes):
    """(start, end) of each line of data, end at its \\n (or the last byte), as file iteration splits them."""
    pos, n = 0, len(data)
    while pos < n:
        nl = data.find(b"\n", pos)
        end = n - 1 if nl < 0 else nl
        yield pos, end
        pos = end + 1


def _read_fasta_bytes(data: bytes):
    """read_fasta over a whole file's bytes: records split at header lines, whitespace
    removed with byte operations (the same records as the line-by-line reader)."""
    if data.startswith(b";") or b"\n;" in data:  # comment lines: the line-by-line reader handles them
        # lines as iterating over the file gives them (split at \n only)
        yield from read_fasta(data[i:j + 1] for i, j in _line_spans(data))
        return
    n = len(data)
    # the first header line; text before it must be whitespace only
    if data.startswith(b">"):
        pos = 0
    else:
        nl = data.find(b"\n>")
        if nl < 0:
            if data.translate(None, _WS):
                raise ValueError("FASTA sequence text before the first header")
            return
        pos = nl + 1
        if data[:pos].translate(None, _WS):
            raise ValueError("FASTA sequence text before the first header")
    while pos < n:
        eol = data.find(b"\n", pos)
        eol = n if eol < 0 else eol
        head = data[pos + 1:eol].strip().split(None, 1)
        nxt = data.find(b"\n>", eol)
        end = n if nxt < 0 else nxt + 1
        name = head[0].decode("utf-8", "replace") if head else ""
        desc = head[1].decode("utf-8", "replace") if len(head) > 1 else ""
        yield Record(name, desc, data[eol:end].translate(None, _WS))
        pos = end


def _nonbase_runs(codes: np.ndarray) -> np.ndarray:
    """[start, length] of each maximal run of code 4 (non-bases), as an (n, 2) uint64 array."""
    bad = np.concatenate(([False], codes == 4, [False]))
    edges = np.flatnonzero(bad[1:] != bad[:-1])
    starts, ends = edges[0::2], edges[1::2]
    return np.stack([starts, ends - starts], axis=1).astype(np.uint64) if len(starts) else np.zeros((0, 2), np.uint64)


def write_bank(path, records) -> dict:
    """Formats records (Record objects, (name, description, sequence) tuples, or a FASTA
    path) into a bank file at path; returns {"n_seqs", "n_bases", "n_runs"}."""
    if isinstance(records, (str, os.PathLike)):
        records = read_fasta(records)
    names, seqs = [], []
    for r in records:
        if not isinstance(r, Record):
            r = Record(*r)
        if "\0" in r.name or "\0" in r.description:
            raise ValueError("names and descriptions cannot hold a 0 byte")
        names.append(r.name.encode() + b"\0" + r.description.encode())
        seqs.append(bytes(r.sequence))
    n = len(seqs)
    seq_start = np.zeros(n + 1, dtype=np.uint64)
    if n:
        seq_start[1:] = np.cumsum([len(s) for s in seqs], dtype=np.uint64)
    text = np.frombuffer(b"".join(seqs), dtype=np.uint8)
    codes = _CODE[text]
    runs = _nonbase_runs(codes)
    c2 = np.where(codes == 4, 0, codes).astype(np.uint8)
    pad = (-len(c2)) % 4
    c2 = np.concatenate([c2, np.zeros(pad, np.uint8)]).reshape(-1, 4)
    packed = (c2[:, 0] << 6) | (c2[:, 1] << 4) | (c2[:, 2] << 2) | c2[:, 3]
    meta_start = np.zeros(n + 1, dtype=np.uint64)
    if n:
        meta_start[1:] = np.cumsum([len(m) for m in names], dtype=np.uint64)
    sections = [seq_start.tobytes(), packed.astype(np.uint8).tobytes(), runs.tobytes(), meta_start.tobytes(),
                b"".join(names)]
    offsets, at = [], _HEADER.size
    for sec in sections:
        at = (at + 7) & ~7
        offsets.append(at)
        at += len(sec)
    with open(path, "wb") as f:
        f.write(_HEADER.pack(MAGIC, VERSION, 0, n, len(text), len(runs), *offsets))
        for off, sec in zip(offsets, sections):
            f.write(b"\0" * (off - f.tell()))
            f.write(sec)
    return {"n_seqs": n, "n_bases": int(len(text)), "n_runs": int(len(runs))}


class BankFile:
    """A formatted bank file, mapped: the metadata is read at open, sequences on demand."""

    def __init__(self, path):
        self.path = os.fspath(path)
        size = os.path.getsize(self.path)
        if size < _HEADER.size:
            raise ValueError("not a bank file (too short)")
        with open(self.path, "rb") as f:
            head = _HEADER.unpack(f.read(_HEADER.size))
        magic, version, _, n, n_bases, n_runs, o_start, o_codes, o_runs, o_meta_start, o_meta = head
        if magic != MAGIC:
            raise ValueError("not a bank file (magic)")
        if version != VERSION:
            raise ValueError(f"bank file version {version}, expected {VERSION}")
        need = [(o_start, 8 * (n + 1)), (o_codes, (n_bases + 3) // 4), (o_runs, 16 * n_runs),
                (o_meta_start, 8 * (n + 1))]
        if any(o + ln > size for o, ln in need):
            raise ValueError("bank file truncated or inconsistent")
        self._map = np.memmap(self.path, dtype=np.uint8, mode="r")
        self.n_seqs, self.n_bases = int(n), int(n_bases)
        self.seq_start = np.array(self._map[o_start:o_start + 8 * (n + 1)].view(np.uint64))
        runs = np.array(self._map[o_runs:o_runs + 16 * n_runs].view(np.uint64)).reshape(-1, 2)
        self._run_start, self._run_len = runs[:, 0], runs[:, 1]
        meta_start = np.array(self._map[o_meta_start:o_meta_start + 8 * (n + 1)].view(np.uint64))
        if self.seq_start[-1] != n_bases or (n and o_meta + int(meta_start[-1]) > size):
            raise ValueError("bank file truncated or inconsistent")
        blob = bytes(self._map[o_meta:o_meta + int(meta_start[-1])])
        self.names, self.descriptions = [], []
        for s in range(n):
            name, _, desc = blob[int(meta_start[s]):int(meta_start[s + 1])].partition(b"\0")
            self.names.append(name.decode())
            self.descriptions.append(desc.decode())
        self._codes_off = o_codes

    def __len__(self) -> int:
        return self.n_seqs

    def _decode(self, a: int, b: int) -> np.ndarray:
        """ASCII of bases [a, b): codes from the file, non-base runs as N."""
        if b <= a:
            return np.zeros(0, dtype=np.uint8)
        lo, hi = a // 4, (b + 3) // 4
        packed = np.asarray(self._map[self._codes_off + lo:self._codes_off + hi])
        codes = np.stack([(packed >> 6) & 3, (packed >> 4) & 3, (packed >> 2) & 3, packed & 3], axis=1).reshape(-1)
        codes = codes[a - 4 * lo:b - 4 * lo].astype(np.uint8)
        # runs that meet [a, b)
        i = int(np.searchsorted(self._run_start, a, side="right")) - 1
        i = max(i, 0)
        while i < len(self._run_start) and int(self._run_start[i]) < b:
            rs, re = int(self._run_start[i]), int(self._run_start[i] + self._run_len[i])
            if re > a:
                codes[max(rs, a) - a:min(re, b) - a] = 4
            i += 1
        return _LETTER[codes]

    def seq(self, s: int) -> bytes:
        """Sequence s (upper-case ACGT, N for non-bases), read from the file."""
        if not 0 <= s < self.n_seqs:
            raise IndexError(s)
        return self._decode(int(self.seq_start[s]), int(self.seq_start[s + 1])).tobytes()

    def arrays(self, chunk: int = 1 << 26):
        """(seq_start, bases) of the whole bank, as ``Index`` takes them (decoded in chunks)."""
        out = np.empty(self.n_bases, dtype=np.uint8)
        for a in range(0, self.n_bases, chunk):
            b = min(self.n_bases, a + chunk)
            out[a:b] = self._decode(a, b)
        return self.seq_start.copy(), out

    def describe(self, s: int) -> str:
        """The header text of sequence s: name and description."""
        return (self.names[s] + " " + self.descriptions[s]).rstrip()
