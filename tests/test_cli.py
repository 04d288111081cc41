"""The command line (text-mode console), on the CPU.

``format`` runs as it is. ``search`` runs its whole host path (bank file, query
FASTA, batching, strands, names, output) with the search itself supplied by the
oracle through the same calls the CUDA library answers, and its output is checked
line by line against the oracle's alignments."""
import os
import xml.etree.ElementTree as ET

import numpy as np

import oracle
import synth
from paper_1507_02987_gb300 import __main__ as cli
from paper_1507_02987_gb300 import bank


class OracleSearch:
    """Stands in for the CUDA library: Index, make_params and search answered by the oracle."""
    GN_FLAG_BOTH_STRANDS = 8

    class Index:
        def __init__(self, start, bases, k=11, stride=11, mask=None):
            self.ox = oracle.Index(synth.Bank(np.asarray(start, np.uint64), np.asarray(bases, np.uint8),
                                              synth.BANKS["tiny"]), k=k, stride=stride, mask=mask)
            self.stride = stride

    @staticmethod
    def make_params(**kw):
        return kw

    class _Res:
        def __init__(self, arrays):
            self.arrays = arrays

        def all(self):
            return self.arrays

        def close(self):
            pass

    def search(self, ix, start, bases, params):
        q = synth.queries_from_strings([bytes(bases[int(start[i]):int(start[i + 1])]) for i in range(len(start) - 1)])
        p = {k: v for k, v in params.items() if k != "flags"}
        both = bool(params.get("flags", 0) & self.GN_FLAG_BOTH_STRANDS)
        res = ix.ox.search(q, oracle.Params(stride=ix.stride, both_strands=both, **p), threads=os.cpu_count() or 1)
        out = []
        for r in res:
            a = np.zeros(len(r.ranked), dtype=[("seq", "<u4"), ("q_start", "<u4"), ("q_end", "<u4"),
                                               ("db_start", "<u4"), ("db_end", "<u4"), ("score", "<i4"),
                                               ("rank", "<u4"), ("evalue", "<f8"), ("bits", "<f8")])
            for fo, fr in (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
                           ("score", "score"), ("rank", "rank"), ("evalue", "evalue"), ("bits", "bits")):
                a[fo] = r.ranked[fr]
            out.append(a)
        return self._Res(out)


def _write_fasta(path, names, seqs, width=60):
    with open(path, "w") as f:
        for n, s in zip(names, seqs):
            f.write(f">{n} some description\n")
            for k in range(0, len(s), width):
                f.write(s[k:k + width].decode() + "\n")


def _case(tmp_path):
    b0 = synth.make_bank("tiny", n_seqs=150)
    qs = synth.make_queries("tiny", b0, n=5)
    bank_fa, q_fa, gnb = tmp_path / "bank.fa", tmp_path / "q.fa", tmp_path / "bank.gnb"
    _write_fasta(bank_fa, [f"chr{i}" for i in range(b0.n_seqs)], [b0.seq(i) for i in range(b0.n_seqs)])
    _write_fasta(q_fa, [f"query_{i}" for i in range(qs.n)], [qs.query(i) for i in range(qs.n)])
    assert cli.main(["format", str(bank_fa), str(gnb)]) == 0
    return b0, qs, gnb, q_fa


def test_format_command(tmp_path):
    b0, qs, gnb, q_fa = _case(tmp_path)
    bf = bank.BankFile(gnb)
    assert len(bf) == b0.n_seqs and bf.names[3] == "chr3" and bf.descriptions[3] == "some description"
    assert bf.seq(7) == b0.seq(7)


def test_search_tsv_matches_the_alignments(tmp_path):
    b0, qs, gnb, q_fa = _case(tmp_path)
    out = tmp_path / "hits.tsv"
    assert cli.main(["search", str(gnb), str(q_fa), "--out", str(out), "--batch", "2"], gn=OracleSearch()) == 0
    lines = out.read_text().splitlines()
    assert lines[0] == cli.TSV_HEADER
    ref = oracle.Index(b0).search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    expect = []
    for i, r in enumerate(ref):
        for h in r.ranked:
            expect.append((f"query_{i}", "+", f"chr{int(h['seq'])}", int(h["score"]), int(h["qs"]) + 1, int(h["qe"]),
                           int(h["ds"]) + 1, int(h["de"]), int(h["rank"]) + 1))
    got = []
    for ln in lines[1:]:
        c = ln.split("\t")
        got.append((c[0], c[1], c[2], int(c[3]), int(c[6]), int(c[7]), int(c[8]), int(c[9]), int(c[10])))
    assert got == expect and len(got) > 0


def test_search_xml_both_strands(tmp_path):
    b0, qs, gnb, q_fa = _case(tmp_path)
    out = tmp_path / "hits.xml"
    assert cli.main(["search", str(gnb), str(q_fa), "--out", str(out), "--format", "xml", "--both-strands",
                     "--max-alignments", "3"], gn=OracleSearch()) == 0
    root = ET.parse(out).getroot()
    qel = root.findall("query")
    assert len(qel) == 2 * qs.n
    assert [q.get("strand") for q in qel[:4]] == ["+", "-", "+", "-"]
    assert all(int(q.get("alignments")) <= 3 for q in qel)
    assert qel[0].get("name") == "query_0" and int(qel[0].get("length")) == len(qs.query(0))
    first = qel[0].find("alignment")
    assert first is not None and first.get("subject").startswith("chr") and first.get("rank") == "1"
