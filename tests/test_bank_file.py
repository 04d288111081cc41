"""The formatted bank file (2-bit sequences with name, identification code and
description, read lazily), on the CPU.

The file keeps what the search uses: a search over the decoded bank gives the
oracle's results over the original FASTA text, whatever its case and non-base
letters."""
import os
import random

import numpy as np
import pytest

import oracle
import synth
from paper_1507_02987_gb300 import bank


def test_read_fasta_forms():
    text = [">gi|1|ref|A1 first sequence, partial\n", "ACGTN\n", "acgu  \n", "\n", "; an old-style comment\n",
            ">two\r\n", "NNNN\r\n", ">three   \n", ">four x  y\n", "RY ACGT\n", "tt\n"]
    recs = list(bank.read_fasta(text))
    assert [(r.name, r.description, r.sequence) for r in recs] == [
        ("gi|1|ref|A1", "first sequence, partial", b"ACGTNacgu"), ("two", "", b"NNNN"), ("three", "", b""),
        ("four", "x  y", b"RYACGTtt")]
    assert list(bank.read_fasta([])) == []
    with pytest.raises(ValueError):
        list(bank.read_fasta(["ACGT\n", ">x\n"]))


def test_round_trip_and_lazy_reads(tmp_path):
    rng = random.Random(5)
    recs = []
    for i in range(60):
        s = "".join(rng.choice("ACGTacgtNnRYKMu") for _ in range(rng.randint(0, 300)))
        recs.append((f"seq{i}", f"description {i}" if i % 3 else "", s.encode()))
    fa = tmp_path / "bank.fa"
    with open(fa, "w") as f:
        for name, desc, s in recs:
            f.write(f">{name} {desc}\n")
            for k in range(0, len(s), 61):
                f.write(s[k:k + 61].decode() + "\n")
    path = tmp_path / "bank.gnb"
    info = bank.write_bank(path, fa)
    assert info["n_seqs"] == 60 and info["n_bases"] == sum(len(s) for _, _, s in recs)
    bf = bank.BankFile(path)
    assert len(bf) == 60
    norm = bytes.maketrans(b"acgtuUnRYKM", b"ACGTTTNNNNN")
    for i in rng.sample(range(60), 60):
        name, desc, s = recs[i]
        assert bf.names[i] == name and bf.descriptions[i] == desc
        assert bf.seq(i) == s.translate(norm)
        assert bf.describe(i) == f"{name} {desc}".rstrip()
    start, bases = bf.arrays(chunk=97)  # chunk edges inside sequences and runs
    assert np.array_equal(start, bf.seq_start)
    assert bases.tobytes() == b"".join(s for _, _, s in recs).translate(norm)
    with pytest.raises(IndexError):
        bf.seq(60)


def test_empty_bank_and_bad_files(tmp_path):
    p = tmp_path / "empty.gnb"
    assert bank.write_bank(p, []) == {"n_seqs": 0, "n_bases": 0, "n_runs": 0}
    bf = bank.BankFile(p)
    assert len(bf) == 0 and bf.arrays()[1].size == 0
    bad = tmp_path / "bad.gnb"
    bad.write_bytes(b"NOTABANK" + bytes(100))
    with pytest.raises(ValueError):
        bank.BankFile(bad)
    good = tmp_path / "good.gnb"
    bank.write_bank(good, [("a", "", b"ACGT" * 100)])
    data = good.read_bytes()
    cut = tmp_path / "cut.gnb"
    cut.write_bytes(data[:100])
    with pytest.raises(ValueError):
        bank.BankFile(cut)
    with pytest.raises(ValueError):
        bank.write_bank(tmp_path / "x.gnb", [("a\0b", "", b"ACGT")])


def test_search_over_decoded_bank_equals_original(tmp_path):
    b0 = synth.make_bank("tiny", n_seqs=200)
    qs = synth.make_queries("tiny", b0, n=6)
    rng = np.random.default_rng(9)
    text = b0.bases.copy()
    # lower case and assorted non-base letters in the bank text
    low = rng.random(len(text)) < 0.2
    text[low] = np.frombuffer(bytes(text[low]).lower(), dtype=np.uint8)
    for ch in b"NRYX":
        text[rng.integers(0, len(text), 40)] = ch
    orig = synth.Bank(b0.seq_start.copy(), text, b0.spec)
    recs = [(f"s{i}", "", orig.seq(i)) for i in range(orig.n_seqs)]
    path = tmp_path / "tiny.gnb"
    bank.write_bank(path, recs)
    start, bases = bank.BankFile(path).arrays()
    decoded = synth.Bank(start, bases, b0.spec)
    r1 = oracle.Index(orig).search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    r2 = oracle.Index(decoded).search(qs, oracle.Params(), threads=os.cpu_count() or 1)
    assert sum(len(r.ranked) for r in r1) > 0
    for a, b in zip(r1, r2):
        assert np.array_equal(a.ranked, b.ranked)


def test_file_reader_equals_line_reader(tmp_path):
    """FASTA files are read as whole bytes; the records equal those of the line-by-line reader."""
    rng = random.Random(17)
    p = tmp_path / "x.fa"
    for trial in range(300):
        parts = []
        if rng.random() < 0.3:
            parts.append(rng.choice(["\n", "  \n", "\r\n", "ACG\n"]))
        for r in range(rng.randint(0, 5)):
            parts.append(">" + rng.choice(["", " ", "name", "n1 desc here", "  spaced  name  x ", "a>b"]) + "\n")
            for line in range(rng.randint(0, 4)):
                parts.append("".join(rng.choice("ACGTacgtN \t>") for _ in range(rng.randint(0, 20)))
                             + rng.choice(["\n", "\r\n"]))
        text = "".join(parts)
        if rng.random() < 0.2:
            text = text.rstrip("\n")
        p.write_text(text)
        try:
            by_line = list(bank.read_fasta(text.splitlines(keepends=True)))
        except ValueError:
            by_line = "error"
        try:
            whole = list(bank.read_fasta(p))
        except ValueError:
            whole = "error"
        assert by_line == whole, repr(text)


def test_fasta_comment_fallback_matches_line_reader(tmp_path):
    """A ';' inside a header does not switch readers; a comment line does, and both readers
    split lines at \\n only (a lone \\r stays inside its line)."""
    text = b">s1 desc;with semicolon\nACGT\rAC\n>s2\nGG\n"
    p = tmp_path / "a.fa"
    p.write_bytes(text)
    with open(p, "rb") as f:
        by_lines = list(bank.read_fasta(f))
    assert list(bank._read_fasta_bytes(text)) == by_lines
    text2 = b";comment\n>s1 d\nAC\r\nGT\n;another\n>s2\nTT\n"
    p.write_bytes(text2)
    with open(p, "rb") as f:
        by_lines = list(bank.read_fasta(f))
    assert list(bank._read_fasta_bytes(text2)) == by_lines
    assert [r.sequence for r in by_lines] == [b"ACGT", b"TT"]
