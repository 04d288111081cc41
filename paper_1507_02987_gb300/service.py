"""HTTP service over the request loop: the paper's web services ("Interfaces": run
queries, set parameters and list the banks from scripts), with the Python standard
library only.

    GET  /banks                   -> [{"name", "sequences", "bases", "k", "stride", "mask"}]
    POST /search?bank=NAME[&max_alignments=N&max_evalue=E&min_hsp_len=L&...]
         body: FASTA text, or JSON {"queries": [{"name", "sequence"}...], "params": {...}}
                                -> {"bank", "queries": [{"name", "length",
                                     "alignments": [{"rank", "subject", "subject_id", "score",
                                                     "bits", "evalue", "q_start", "q_end",
                                                     "s_start", "s_end"}]}]}

Each bank has one request loop (``Server``: continuous batching over the resident
index, admission by memory footprint); every query of a request is submitted to it
and the results are collected by ticket, so concurrent requests share micro-batches.
Search parameters (``PARAMS``: hit distance, minimum HSP length, drop-off, number of
alignments, band half-width, e-value cut) may be set per request, in the query
string or the JSON body.  Each is checked (an integer, or a number for the e-value
cut, inside the library's range; 400 otherwise) and completed with the library's
defaults, so a request that names the default values shares the default loop.  Each
distinct set gets a request loop of its own, at most ``max_param_sets`` per bank; the
bank's memory budget is split evenly across them, so that the device never holds more
than that budget for the bank.  When a new set needs a loop and all are taken, the
least recently used set with no request in flight is stopped and replaced (503 if
every set is busy). Queries are
searched on the strand given (``gn_search`` with ``GN_FLAG_BOTH_STRANDS``, or the
command line's ``--both-strands``, searches both).
Ranges are 0-based and end-exclusive, as in the library's results.
"""
from __future__ import annotations

import json
import math
import threading
import time
from http.server import BaseHTTPRequestHandler, ThreadingHTTPServer
from urllib.parse import parse_qs, urlparse

from . import bank as bankmod


# per-request search parameters: name -> (type, smallest, largest) as the library takes them
PARAMS = {"max_hit_distance": (int, 0, 65535), "min_hsp_len": (int, 0, 2**32 - 1), "xdrop": (int, 0, 2**31 - 1),
          "max_alignments": (int, 0, 2**32 - 1), "band_w": (int, 0, 16384), "max_evalue": (float, 0.0, math.inf)}


class Busy(Exception):
    """Every request loop of the bank is in use by another parameter set."""


def check_param(name, value):
    """The value of a search parameter as the library takes it; ValueError if it is not."""
    if name not in PARAMS:
        raise ValueError(f"unknown parameter {name!r}")
    kind, lo, hi = PARAMS[name]
    if isinstance(value, bool):
        raise ValueError(f"{name}: {value!r} is not a number")
    try:
        x = float(value)
    except (TypeError, ValueError):
        raise ValueError(f"{name}: {value!r} is not a number") from None
    if math.isnan(x) or not lo <= x <= hi:
        raise ValueError(f"{name}: {value!r} is outside [{lo}, {hi}]")
    if kind is int:
        if not x.is_integer():
            raise ValueError(f"{name}: {value!r} is not an integer")
        return int(x)
    return x


class BankService:
    """One served bank: its metadata, its index and a request loop per parameter set."""

    def __init__(self, gn, name, bank_file, mem_budget, index=None, k=11, stride=11, mask=None,
                 max_param_sets=4):
        self.gn, self.name = gn, name
        self.bf = bank_file if isinstance(bank_file, bankmod.BankFile) else bankmod.BankFile(bank_file)
        if index is None:
            start, bases = self.bf.arrays()
            index = gn.Index(start, bases, k=k, stride=stride, mask=mask)
        self.index = index
        self.k, self.stride, self.mask = k, stride, mask
        self.mem_budget, self.max_param_sets = mem_budget, max_param_sets
        # the library's defaults, with the hit distance and minimum HSP length resolved
        self.defaults = {"max_hit_distance": 3 * stride, "min_hsp_len": 2 * (mask.count("1") if mask else k),
                         "xdrop": 20, "max_alignments": 100, "band_w": 16, "max_evalue": math.inf}
        self.default_key = self.key_of({})
        self.servers = {self.default_key: gn.Server(index, self.loop_budget())}
        self.in_flight = {self.default_key: 0}
        self.last_use = {self.default_key: 0.0}
        self.lock = threading.Lock()

    def loop_budget(self) -> int:
        return max(1, self.mem_budget // self.max_param_sets)

    def key_of(self, params: dict) -> tuple:
        """The complete, checked parameter set of a request (defaults filled in)."""
        full = dict(self.defaults)
        for name, value in params.items():
            full[name] = check_param(name, value)
        if full["max_hit_distance"] == 0:
            full["max_hit_distance"] = self.defaults["max_hit_distance"]
        if full["min_hsp_len"] == 0:
            full["min_hsp_len"] = self.defaults["min_hsp_len"]
        return tuple(sorted(full.items()))

    def acquire(self, params: dict):
        """(key, request loop) of a parameter set, created on first use; the caller releases it."""
        key = self.key_of(params)
        with self.lock:
            srv = self.servers.get(key)
            if srv is None:
                if len(self.servers) >= self.max_param_sets:
                    idle = [k for k in self.servers if k != self.default_key and self.in_flight[k] == 0]
                    if not idle:
                        raise Busy(f"all {self.max_param_sets} parameter sets of this bank are in use")
                    old = min(idle, key=lambda k: self.last_use[k])
                    self.servers.pop(old).stop()
                    del self.in_flight[old], self.last_use[old]
                srv = self.gn.Server(self.index, self.loop_budget(), params=self.gn.make_params(**dict(key)))
                self.servers[key] = srv
                self.in_flight[key] = 0
            self.in_flight[key] += 1
            self.last_use[key] = time.monotonic()
            return key, srv

    def release(self, key):
        with self.lock:
            if key in self.in_flight:
                self.in_flight[key] -= 1

    def describe(self) -> dict:
        return {"name": self.name, "sequences": self.bf.n_seqs, "bases": self.bf.n_bases, "k": self.k,
                "stride": self.stride, "mask": self.mask}

    def search(self, queries, params=None, timeout_ms=600000) -> dict:
        """queries: [(name, sequence bytes)]; one result entry per query, in order."""
        key, srv = self.acquire(params or {})
        try:
            jobs = [(name, seq, srv.submit(seq)) for name, seq in queries]
            out = []
            for name, seq, ticket in jobs:
                res = srv.poll(ticket, timeout_ms)
                if res is None:
                    raise TimeoutError(f"query {name} did not finish")
                hits = res.query(0)
                res.close()
                out.append({"name": name, "length": len(seq), "alignments": [
                    {"rank": int(h["rank"]) + 1, "subject": self.bf.names[int(h["seq"])],
                     "subject_id": int(h["seq"]), "score": int(h["score"]), "bits": float(h["bits"]),
                     "evalue": float(h["evalue"]), "q_start": int(h["q_start"]), "q_end": int(h["q_end"]),
                     "s_start": int(h["db_start"]), "s_end": int(h["db_end"])} for h in hits]})
        finally:
            self.release(key)
        return {"bank": self.name, "queries": out}

    def close(self):
        for srv in self.servers.values():
            srv.stop()


def parse_queries(body: bytes, content_type: str):
    """([(name, sequence)], params) from a FASTA body or a JSON {"queries": [...], "params": {...}} body."""
    if content_type.startswith("application/json") or body.lstrip()[:1] == b"{":
        doc = json.loads(body)
        qs = [(str(q.get("name", f"q{i}")), str(q["sequence"]).encode()) for i, q in enumerate(doc["queries"])]
        return qs, dict(doc.get("params", {}))
    return [(r.name, r.sequence) for r in bankmod.read_fasta(body.decode("utf-8", "replace").splitlines())], {}


def make_handler(banks: dict):
    class Handler(BaseHTTPRequestHandler):
        def _send(self, code, doc):
            data = json.dumps(doc).encode()
            self.send_response(code)
            self.send_header("Content-Type", "application/json")
            self.send_header("Content-Length", str(len(data)))
            self.end_headers()
            self.wfile.write(data)

        def log_message(self, fmt, *args):  # quiet
            pass

        def do_GET(self):
            if urlparse(self.path).path == "/banks":
                return self._send(200, [b.describe() for b in banks.values()])
            return self._send(404, {"error": "unknown path"})

        def do_POST(self):
            url = urlparse(self.path)
            if url.path != "/search":
                return self._send(404, {"error": "unknown path"})
            qs = parse_qs(url.query)
            name = qs.get("bank", [next(iter(banks), "")])[0]
            if name not in banks:
                return self._send(404, {"error": f"no bank {name!r}"})
            try:
                body = self.rfile.read(int(self.headers.get("Content-Length", "0")))
                queries, params = parse_queries(body, self.headers.get("Content-Type", ""))
                params.update({k: v[0] for k, v in qs.items() if k != "bank"})
                return self._send(200, banks[name].search(queries, params))
            except (ValueError, KeyError, json.JSONDecodeError) as e:
                return self._send(400, {"error": str(e)})
            except Busy as e:
                return self._send(503, {"error": str(e)})
            except Exception as e:  # a library error: the status and message of the call
                return self._send(500, {"error": str(e)})

    return Handler


def serve(banks: dict, host="127.0.0.1", port=8080):
    """Starts the HTTP service on a background thread; returns (server, thread). server.shutdown() stops it."""
    httpd = ThreadingHTTPServer((host, port), make_handler(banks))
    th = threading.Thread(target=httpd.serve_forever, daemon=True)
    th.start()
    return httpd, th
