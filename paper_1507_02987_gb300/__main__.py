"""Command line: the paper's text-mode console ("Interfaces": batch searches from
the console with the results written out), over the C ABI.

    python -m paper_1507_02987_gb300 format BANK.fa BANK.gnb
    python -m paper_1507_02987_gb300 index BANK.gnb BANK.gnx [--k 11] [--stride 11] [--mask M]
    python -m paper_1507_02987_gb300 serve BANK.gnb [--index BANK.gnx] [--port 8080] [--budget-gib 16]
    python -m paper_1507_02987_gb300 search BANK.gnb QUERIES.fa [--index BANK.gnx | --k/--stride/--mask]
                                         [--out FILE] [--format tsv|xml] [--both-strands]
                                         [--max-alignments N] [--max-evalue E] [--band-w W] ...

``format`` runs on the host. ``index``, ``search`` and ``serve`` (the HTTP service
of ``service.py``) need the CUDA library and a GPU; there is no CPU fallback. ``search`` sends the queries in calls of at most
``--batch`` queries and writes one line (tsv) or element (xml) per alignment in
rank order: query name, strand, bank sequence name, score, bit score, e-value and
1-based inclusive ranges (on the reverse complement of the query for the minus
strand)."""
from __future__ import annotations

import argparse
import sys
from xml.sax.saxutils import quoteattr

import numpy as np

from . import bank as bankmod

TSV_HEADER = "query\tstrand\tsubject\tscore\tbits\tevalue\tq_start\tq_end\ts_start\ts_end\trank"


def _rows(query_names, query_lens, subject_names, results, both_strands):
    """(query name, query length, strand, hit records) per result query."""
    for i, hits in enumerate(results):
        q = i // 2 if both_strands else i
        strand = "-" if both_strands and i % 2 else "+"
        yield query_names[q], query_lens[q], strand, hits


def format_tsv(query_names, query_lens, subject_names, results, both_strands=False) -> str:
    """Tab-separated alignments, one per line, after a header line."""
    out = [TSV_HEADER]
    for qn, _, strand, hits in _rows(query_names, query_lens, subject_names, results, both_strands):
        for h in hits:
            out.append(f"{qn}\t{strand}\t{subject_names[int(h['seq'])]}\t{int(h['score'])}\t{float(h['bits']):.1f}\t"
                       f"{float(h['evalue']):.3g}\t{int(h['q_start']) + 1}\t{int(h['q_end'])}\t"
                       f"{int(h['db_start']) + 1}\t{int(h['db_end'])}\t{int(h['rank']) + 1}")
    return "\n".join(out) + "\n"


def format_xml(query_names, query_lens, subject_names, results, both_strands=False) -> str:
    """The same alignments as an XML document."""
    out = ['<?xml version="1.0" encoding="UTF-8"?>', "<results>"]
    for qn, ql, strand, hits in _rows(query_names, query_lens, subject_names, results, both_strands):
        out.append(f"  <query name={quoteattr(qn)} length=\"{ql}\" strand=\"{strand}\" alignments=\"{len(hits)}\">")
        for h in hits:
            out.append(f"    <alignment rank=\"{int(h['rank']) + 1}\" subject={quoteattr(subject_names[int(h['seq'])])} "
                       f"score=\"{int(h['score'])}\" bits=\"{float(h['bits']):.1f}\" "
                       f"evalue=\"{float(h['evalue']):.3g}\" q_start=\"{int(h['q_start']) + 1}\" "
                       f"q_end=\"{int(h['q_end'])}\" s_start=\"{int(h['db_start']) + 1}\" "
                       f"s_end=\"{int(h['db_end'])}\"/>")
        out.append("  </query>")
    out.append("</results>")
    return "\n".join(out) + "\n"


def _build_index(gn, bf, args):
    start, bases = bf.arrays()
    return gn.Index(start, bases, k=args.k, stride=args.stride, mask=args.mask)


def run_search(gn, args) -> str:
    """Searches the query FASTA against the bank; returns the formatted output."""
    bf = bankmod.BankFile(args.bank)
    ix = gn.Index.load(args.index) if args.index else _build_index(gn, bf, args)
    recs = list(bankmod.read_fasta(args.queries))
    names = [r.name for r in recs]
    lens = [len(r.sequence) for r in recs]
    flags = gn.GN_FLAG_BOTH_STRANDS if args.both_strands else 0
    params = gn.make_params(max_hit_distance=args.max_hit_distance, min_hsp_len=args.min_hsp_len, xdrop=args.xdrop,
                            max_alignments=args.max_alignments, band_w=args.band_w, max_evalue=args.max_evalue,
                            flags=flags)
    results = []
    for a in range(0, len(recs), args.batch):
        part = recs[a:a + args.batch]
        start = np.zeros(len(part) + 1, dtype=np.uint64)
        start[1:] = np.cumsum([len(r.sequence) for r in part])
        bases = np.frombuffer(b"".join(r.sequence for r in part), dtype=np.uint8)
        res = gn.search(ix, start, bases, params=params)
        results.extend(res.all())
        res.close()
    fmt = format_xml if args.format == "xml" else format_tsv
    return fmt(names, lens, bf.names, results, args.both_strands)


def main(argv=None, gn=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1507_02987_gb300")
    sub = ap.add_subparsers(dest="cmd", required=True)
    f = sub.add_parser("format", help="FASTA bank -> formatted bank file")
    f.add_argument("fasta")
    f.add_argument("out")
    for name in ("index", "search", "serve"):
        p = sub.add_parser(name)
        p.add_argument("bank", help="formatted bank file")
        if name == "index":
            p.add_argument("out", help="index file to write")
        elif name == "serve":
            p.add_argument("--index", help="a saved index of this bank (else one is built)")
            p.add_argument("--host", default="127.0.0.1")
            p.add_argument("--port", type=int, default=8080)
            p.add_argument("--budget-gib", type=float, default=16.0, help="request loop memory budget")
        else:
            p.add_argument("queries", help="query FASTA")
            p.add_argument("--index", help="a saved index of this bank (else one is built)")
            p.add_argument("--out", help="output file (default: standard output)")
            p.add_argument("--format", choices=["tsv", "xml"], default="tsv")
            p.add_argument("--both-strands", action="store_true")
            p.add_argument("--max-hit-distance", type=int, default=0, help="0: 3 x stride")
            p.add_argument("--min-hsp-len", type=int, default=0, help="0: 2 x k")
            p.add_argument("--xdrop", type=int, default=20)
            p.add_argument("--max-alignments", type=int, default=100, help="per query; 0: all")
            p.add_argument("--band-w", type=int, default=16)
            p.add_argument("--max-evalue", type=float, default=float("inf"))
            p.add_argument("--batch", type=int, default=4096, help="queries per search call")
        p.add_argument("--k", type=int, default=11)
        p.add_argument("--stride", type=int, default=11)
        p.add_argument("--mask", default=None, help="spaced seed, e.g. 111010010100110111")
    args = ap.parse_args(argv)
    if args.cmd == "format":
        info = bankmod.write_bank(args.out, args.fasta)
        print(f"{info['n_seqs']} sequences, {info['n_bases']} bases, {info['n_runs']} non-base runs -> {args.out}",
              file=sys.stderr)
        return 0
    if gn is None:
        import paper_1507_02987_gb300 as gn
        gn.load()
    if args.cmd == "index":
        ix = _build_index(gn, bankmod.BankFile(args.bank), args)
        ix.save(args.out)
        ix.close()
        return 0
    if args.cmd == "serve":
        import os
        import time

        from . import service
        bf = bankmod.BankFile(args.bank)
        ix = gn.Index.load(args.index) if args.index else _build_index(gn, bf, args)
        name = os.path.splitext(os.path.basename(args.bank))[0]
        svc = service.BankService(gn, name, bf, int(args.budget_gib * 2**30), index=ix, k=args.k,
                                  stride=args.stride, mask=args.mask)
        httpd, _ = service.serve({name: svc}, args.host, args.port)
        print(f"serving bank {name!r} on http://{args.host}:{httpd.server_address[1]}", file=sys.stderr)
        try:
            while True:
                time.sleep(3600)
        except KeyboardInterrupt:
            httpd.shutdown()
            svc.close()
        return 0
    text = run_search(gn, args)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    else:
        sys.stdout.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
