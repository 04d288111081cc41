"""The HTTP service (web-service interface) on the CPU.

The request loop is stood in for by the oracle behind the same submit / poll calls,
so the test covers the service's whole host path: bank listing, FASTA and JSON
request bodies, concurrent requests, names and error statuses."""
import json
import os
import threading
import urllib.error
import urllib.request

import numpy as np
import pytest

import oracle
import synth
from paper_1507_02987_gb300 import bank, service


class _Res:
    def __init__(self, arr):
        self.arr = arr

    def query(self, i):
        assert i == 0
        return self.arr

    def close(self):
        pass


class OracleLoop:
    """submit / poll / stop of the request loop, answered by the oracle."""
    GN_FLAG_BOTH_STRANDS = 8

    class Index:
        def __init__(self, start, bases, k=11, stride=11, mask=None):
            self.ox = oracle.Index(synth.Bank(np.asarray(start, np.uint64), np.asarray(bases, np.uint8),
                                              synth.BANKS["tiny"]), k=k, stride=stride, mask=mask)

    @staticmethod
    def make_params(**kw):
        return kw

    class Server:
        def __init__(self, index, budget, params=None):
            self.index, self.done, self.lock, self.next = index, {}, threading.Lock(), 0
            self.params = params or {}

        def submit(self, seq):
            r = self.index.ox.search([bytes(seq)], oracle.Params(**self.params))[0].ranked
            a = np.zeros(len(r), dtype=[("seq", "<u4"), ("q_start", "<u4"), ("q_end", "<u4"), ("db_start", "<u4"),
                                        ("db_end", "<u4"), ("score", "<i4"), ("rank", "<u4"), ("evalue", "<f8"),
                                        ("bits", "<f8")])
            for fo, fr in (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
                           ("score", "score"), ("rank", "rank"), ("evalue", "evalue"), ("bits", "bits")):
                a[fo] = r[fr]
            with self.lock:
                t = self.next
                self.next += 1
                self.done[t] = a
            return t

        def poll(self, ticket, timeout_ms):
            with self.lock:
                a = self.done.pop(ticket, None)
            return None if a is None else _Res(a)

        def stop(self):
            pass


@pytest.fixture(scope="module")
def running(tmp_path_factory):
    d = tmp_path_factory.mktemp("svc")
    b0 = synth.make_bank("tiny", n_seqs=150)
    qs = synth.make_queries("tiny", b0, n=4)
    gnb = d / "tiny.gnb"
    bank.write_bank(gnb, [(f"chr{i}", "d", b0.seq(i)) for i in range(b0.n_seqs)])
    svc = service.BankService(OracleLoop(), "tiny", str(gnb), 1 << 30)
    httpd, _ = service.serve({"tiny": svc}, "127.0.0.1", 0)
    url = f"http://127.0.0.1:{httpd.server_address[1]}"
    yield b0, qs, url
    httpd.shutdown()
    svc.close()


def _post(url, body, ctype):
    req = urllib.request.Request(url, data=body, headers={"Content-Type": ctype}, method="POST")
    with urllib.request.urlopen(req, timeout=60) as r:
        return json.loads(r.read())


def test_list_banks(running):
    b0, qs, url = running
    with urllib.request.urlopen(url + "/banks", timeout=30) as r:
        doc = json.loads(r.read())
    assert doc == [{"name": "tiny", "sequences": b0.n_seqs, "bases": b0.n_bases, "k": 11, "stride": 11,
                    "mask": None}]


def test_search_fasta_and_json_bodies(running):
    b0, qs, url = running
    ref = oracle.Index(b0).search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    fasta = "".join(f">q{i} x\n{qs.query(i).decode()}\n" for i in range(qs.n)).encode()
    doc = _post(url + "/search?bank=tiny", fasta, "text/plain")
    doc2 = _post(url + "/search", json.dumps({"queries": [{"name": f"q{i}", "sequence": qs.query(i).decode()}
                                                           for i in range(qs.n)]}).encode(), "application/json")
    assert doc == doc2 and doc["bank"] == "tiny" and len(doc["queries"]) == qs.n
    for i, q in enumerate(doc["queries"]):
        assert q["name"] == f"q{i}" and q["length"] == len(qs.query(i))
        got = [(a["subject"], a["score"], a["q_start"], a["q_end"], a["s_start"], a["s_end"], a["rank"])
               for a in q["alignments"]]
        exp = [(f"chr{int(h['seq'])}", int(h["score"]), int(h["qs"]), int(h["qe"]), int(h["ds"]), int(h["de"]),
                int(h["rank"]) + 1) for h in ref[i].ranked]
        assert got == exp
    assert sum(len(q["alignments"]) for q in doc["queries"]) > 0


def test_concurrent_requests_and_errors(running):
    b0, qs, url = running
    out = {}

    def client(i):
        out[i] = _post(url + "/search", f">only\n{qs.query(i).decode()}\n".encode(), "text/plain")

    ths = [threading.Thread(target=client, args=(i,)) for i in range(qs.n)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for i in range(qs.n):
        assert out[i]["queries"][0]["length"] == len(qs.query(i))
    for path, body, code in (("/search?bank=nope", b">a\nACGT\n", 404), ("/nowhere", b"", 404),
                             ("/search", b"ACGT without a header", 400), ("/search", b"{\"queries\": [{}]}", 400)):
        with pytest.raises(urllib.error.HTTPError) as e:
            _post(url + path, body, "text/plain")
        assert e.value.code == code


def test_parameters_per_request(running):
    b0, qs, url = running
    fasta = "".join(f">q{i}\n{qs.query(i).decode()}\n" for i in range(qs.n)).encode()
    doc = _post(url + "/search?max_alignments=2&xdrop=10", fasta, "text/plain")
    ref = oracle.Index(b0).search(qs, oracle.Params(max_alignments=2, xdrop=10), threads=os.cpu_count() or 1)
    for i, q in enumerate(doc["queries"]):
        assert len(q["alignments"]) == len(ref[i].ranked) <= 2
        assert [a["score"] for a in q["alignments"]] == [int(h["score"]) for h in ref[i].ranked]
    body = json.dumps({"queries": [{"name": "a", "sequence": qs.query(0).decode()}],
                       "params": {"max_alignments": 1}}).encode()
    assert len(_post(url + "/search", body, "application/json")["queries"][0]["alignments"]) <= 1
    for path in ("/search?no_such=1", "/search?max_alignments=x"):
        with pytest.raises(urllib.error.HTTPError) as e:
            _post(url + path, fasta, "text/plain")
        assert e.value.code == 400
    # the default set and three more fill the pool of four: a fifth set replaces the least
    # recently used idle one, and its results are still right
    _post(url + "/search?max_alignments=3", fasta, "text/plain")
    doc = _post(url + "/search?max_alignments=4", fasta, "text/plain")
    ref = oracle.Index(b0).search(qs, oracle.Params(max_alignments=4), threads=os.cpu_count() or 1)
    assert [len(q["alignments"]) for q in doc["queries"]] == [len(r.ranked) for r in ref]


def test_parameter_sets_share_loops_and_are_checked(tmp_path):
    b0 = synth.make_bank("tiny", n_seqs=60)
    gnb = tmp_path / "t.gnb"
    bank.write_bank(gnb, [(f"chr{i}", "d", b0.seq(i)) for i in range(b0.n_seqs)])
    svc = service.BankService(OracleLoop(), "t", str(gnb), 1 << 30, max_param_sets=2)
    q = [("a", synth.make_queries("tiny", b0, n=1).query(0))]
    # the library's default values, named or left out, are one set: the default loop
    for params in ({}, {"band_w": 16}, {"max_alignments": 100, "xdrop": "20"}, {"max_hit_distance": 33},
                   {"min_hsp_len": 22}, {"max_evalue": "inf"}, {"band_w": 16.0}):
        svc.search(q, params)
        assert len(svc.servers) == 1, params
    # each loop gets an even share of the bank's budget
    assert svc.loop_budget() == (1 << 30) // 2
    # out of range, negative, fractional or non-numeric values are refused
    for params in ({"max_alignments": -1}, {"min_hsp_len": -5}, {"max_alignments": 2.7}, {"band_w": 16385},
                   {"xdrop": "x"}, {"max_evalue": -1}, {"max_hit_distance": 70000}, {"band_w": True},
                   {"max_evalue": "nan"}):
        with pytest.raises(ValueError):
            svc.search(q, params)
    # a second set takes the second loop; a third replaces it (least recently used, idle)
    svc.search(q, {"max_alignments": 5})
    svc.search(q, {"max_alignments": 6})
    assert len(svc.servers) == 2 and svc.default_key in svc.servers
    # with every non-default loop busy, a new set is refused
    key, _ = svc.acquire({"max_alignments": 6})
    with pytest.raises(service.Busy):
        svc.search(q, {"max_alignments": 7})
    svc.release(key)
    svc.search(q, {"max_alignments": 7})
    svc.close()
