#!/usr/bin/env python3
"""Throughput benchmark of the Genoogle search path on GB300.

Metric: query kbp/s (query bases searched per second, in thousands) against the
~4 Gbp synthetic bank, index resident in device memory.  One step = one
gn_search call over the whole query set of the workload (2,000 queries of
200-20,000 bp for the default `large` workload), i.e. every phase of the
search: query codes, seed gather, hit sort, hit merge, X-drop extension,
overlap merge, selection, banded Smith-Waterman, ranking.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs as N independent replicas under torchrun (one bank, index and query
set per rank; no data exchange), reported as weak scaling.  `--impl reference`
times the CPU oracle (the plain C implementation used as the correctness
reference) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query kbp/s vs 4 Gbp bank (batched/served vs plain, same GPU); p50/p99 latency"
UNIT = "kbp/s"

# Algorithmic bytes per work item of each kernel (HBM-bound kernels), see the design notes:
#   sort pass (or downsweep): read + write one 8-byte key (and a 4-byte value); histogram (or
#   upsweep): read the key
#   seed gather: read one 4-byte occurrence, write one 8-byte hit key
#   hit merge: read one 8-byte hit key
BYTES_PER_UNIT = {
    "hit_sort_pass": 16.0,
    "hit_sort_hist": 8.0,
    "hit_sort_downsweep": 16.0,
    "hit_sort_upsweep": 8.0,
    "k_seed_gather": 12.0,
    "k_hit_merge": 8.0,
    "record_sort_pass": 24.0,
    "record_sort_hist": 8.0,
    "record_sort_downsweep": 24.0,
    "record_sort_upsweep": 8.0,
    "k_query_codes": 17.0,
    # bucket fill (units = hits): one 4-byte occurrence read per hit; the 8-byte writes of the
    # kept hits are added from k_bucket_group's units (kept hits) in roofline()
    "k_bucket_fill": 4.0,
    "k_bucket_group": 8.0,   # units = kept hits: one 8-byte bucket entry read
}
# integer-ALU kernels: units = DP cells of the band area; 8 algorithmic integer operations per
# cell (E and F: add + max each; H: substitution select, add, three-way max with 0)
ALU_KERNELS = {"k_banded_sw", "k_banded_sw_wide"}
ALU_OPS_PER_UNIT = 8.0
# their peak: integer operations per second measured in the same run by gn_measure_int_peaks
# (DPX add-max, two operations per instruction, every SM filled)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large", choices=["tiny", "mid", "batched", "large", "long"])
    ap.add_argument("--stride", type=int, default=11)
    ap.add_argument("--mask", default=None, help="spaced-seed mask, e.g. 111010010100110111 (k = its ones)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the band width and kernel tuning on a 200-query calibration sample first")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-queries", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target oracle time of the CPU baseline")
    ap.add_argument("--queries", type=int, default=0, help="use only the first N queries (profiling runs)")
    ap.add_argument("--serve-rates", default="50,200,2000,max",
                    help="Poisson arrival rates (queries/s) of the serving leg ('max': every request arrives "
                         "at once, a saturation run of all requests); empty to skip it")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="arrival window per serving rate")
    ap.add_argument("--serve-budget-gib", type=float, default=16.0, help="server memory budget")
    ap.add_argument("--no-sub-legs", action="store_true",
                    help="skip the batched (10,000 queries on the mid bank) and long-query sub-legs")
    ap.add_argument("--sweep", action="store_true",
                    help="sensitivity sweep instead of the benchmark: planted-homolog recovery and time per "
                         "step for a grid of minimum HSP length, hit distance and drop-off around the defaults")
    return ap.parse_args()


# ------------------------------------------------------------- plumbing --
class Dist:
    def __init__(self):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group(backend="gloo")  # host-side barrier and timing reduction only
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(device_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "", 1).isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def csrc_digest() -> str:
    """Digest of the device-code sources (every csrc file but the host-only C ABI file,
    which holds no kernel): committed ncu traffic counts are valid while it is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1507_02987_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f == "gn_abi.cu":
            continue
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per work item of `kernel` from the committed ncu summary, if it is current."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except Exception:
        return None
    if t.get("csrc_digest") != csrc_digest():
        return None
    k = t.get("kernels", {}).get(kernel)
    return k.get("dram_bytes_per_unit") if k else None


def workload_desc(name: str, stride: int) -> str:
    desc = {
        "tiny": "tiny bank (1,000 uniform sequences, ~1.25 Mbp), 10 mutated-copy queries",
        "mid": "mid bank (200,000 log-normal sequences, ~400 Mbp, GC 0.35-0.65, 20% repeats), 1,000 homolog queries 80-10,000 bp",
        "batched": "mid bank (~400 Mbp), 10,000 queries 50-5,000 bp, half planted homologs",
        "large": "large bank (2.5 M log-normal sequences, ~4.0 Gbp, GC 0.35-0.65, 20% repeats), 2,000 queries 200-20,000 bp, half planted homologs",
        "long": "large bank (~4.0 Gbp), 40 queries 65,536 bp - 1 Mbp (searched in overlapping segments), half planted homologs",
    }[name]
    return f"{desc}; k=11, stride {stride}; one gn_search over all queries per step"


def workload(name: str, stride: int, rank: int, n_queries: int = 0):
    import dataclasses

    import numpy as np
    import synth
    import torch

    pinned = lambda n: torch.empty(int(n), dtype=torch.uint8, pin_memory=True).numpy()
    bank = synth.make_bank(name, alloc=pinned if torch.cuda.is_available() else None)
    spec = synth.QUERIES[name]
    if rank:
        spec = dataclasses.replace(spec, seed=spec.seed + 1000 * rank)
    queries = synth.make_queries(spec, bank)
    if n_queries and n_queries < queries.n:
        queries = queries.subset(range(n_queries))
    return bank, queries, workload_desc(name, stride)


def oracle_run(bank, queries, stride, threads, target_s, rng_seed=0, mask=None, band_w=16):
    """Times the oracle on growing samples of the query set until one takes >= target_s/2; returns
    (kbp/s, seconds, sample description, sample indices, results)."""
    import oracle
    ox = oracle.Index(bank, k=11, stride=stride, mask=mask)
    n = min(queries.n, 16)
    order = list(range(0, queries.n, max(1, queries.n // 997)))
    while True:
        idx = order[:n] if n <= len(order) else list(range(min(n, queries.n)))
        sub = queries.subset(idx)
        t0 = time.perf_counter()
        res = ox.search(sub, oracle.Params(stride=stride, band_w=band_w), threads=threads)
        dt = time.perf_counter() - t0
        if dt >= target_s / 2 or n >= queries.n:
            bases = int(sub.start[-1])
            return bases / 1e3 / dt, dt, (f"{len(idx)} of {queries.n} queries (evenly spaced), {bases} bases, "
                                          f"all {threads} host threads, index resident"), idx, res, ox
        n = min(queries.n, max(n + 1, int(n * min(8.0, max(2.0, target_s / max(dt, 1e-3))))))


def percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def same_result(a, b):
    """Two one-query results agree: integers identical, e-values within 1e-9 relative (both below
    1e-300 counts as equal)."""
    import numpy as np
    if a is None or b is None or len(a) != len(b):
        return False
    for f in ("seq", "q_start", "q_end", "db_start", "db_end", "score", "rank"):
        if not np.array_equal(a[f], b[f]):
            return False
    tiny = (np.abs(a["evalue"]) < 1e-300) & (np.abs(b["evalue"]) < 1e-300)
    return bool((tiny | np.isclose(a["evalue"], b["evalue"], rtol=1e-9, atol=0)).all())


def serve_leg(gn, ix, reqs, arrivals, budget, timeout_s=120.0):
    """Open-loop run of the request loop: submits reqs[i] at t0 + arrivals[i], collects results from
    the completion queue on another thread.  Latency = result on the host - scheduled arrival.
    Returns the leg's figures and each request's result (read after the run)."""
    srv = gn.Server(ix, budget)
    n = len(reqs)
    done_at = {}
    held = {}  # ticket -> result, read and freed after the run: the collector does as little as it can

    def collector():
        end = time.perf_counter() + timeout_s
        while len(done_at) < n and time.perf_counter() < end:
            got = srv.poll_any(200)
            if got is None:
                continue
            done_at[got[0]] = time.perf_counter()
            held[got[0]] = got[1]

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    tickets = []
    for i in range(n):
        wait = t0 + float(arrivals[i]) - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(reqs[i]))
    submit_s = time.perf_counter() - t0
    th.join(timeout_s)
    results = [held[t].query(0).copy() if t in held else None for t in tickets]
    for res in held.values():
        res.close()
    stats = srv.stats()
    srv.stop()
    lat = [1e3 * (done_at[t] - (t0 + float(arrivals[i]))) for i, t in enumerate(tickets) if t in done_at]
    wall = (max(done_at.values()) - t0) if done_at else float("nan")
    return {"requests": n, "completed": len(lat), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
            "kbp_s": sum(len(r) for r in reqs) / 1e3 / wall, "batches": stats["batches"],
            "max_batch": stats["max_batch"], "max_concurrent_batches": stats["max_concurrent"],
            "submit_ms": 1e3 * submit_s}, results


def plain_leg(gn, ix, reqs, arrivals, stream):
    """The same arrivals served by the plain path: one gn_search per query, in arrival order, with host
    queries and host results.  Returns the leg's figures and each request's result."""
    import numpy as np
    t0 = time.perf_counter()
    lat, results = [], []
    for i, q in enumerate(reqs):
        wait = t0 + float(arrivals[i]) - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        st = np.array([0, len(q)], dtype=np.uint64)
        res = gn.search(ix, st, np.frombuffer(q, dtype=np.uint8), stream=stream)
        results.append(res.query(0).copy())
        res.close()
        lat.append(1e3 * (time.perf_counter() - (t0 + float(arrivals[i]))))
    wall = time.perf_counter() - t0
    return {"requests": len(reqs), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
            "kbp_s": sum(len(r) for r in reqs) / 1e3 / wall}, results


def serving(args, gn, ix, bank, stream, log):
    """Serving leg: open-loop Poisson arrivals of the serving request mix against the resident index,
    through the request loop and through the plain path, at each rate."""
    import numpy as np
    import synth
    rates = [r.strip() for r in args.serve_rates.split(",") if r.strip()]
    if not rates or args.workload != "large":
        return None
    spec = synth.QUERIES["serving"]
    qs = synth.make_queries(spec, bank)
    reqs = [qs.query(i) for i in range(qs.n)]
    budget = int(args.serve_budget_gib * 2**30)
    out = {"requests_from": f"{qs.n} requests, log-uniform 50-20,000 bp, 30% planted homologs",
           "budget_gib": args.serve_budget_gib, "rates": []}
    for r in rates:
        if r == "max":
            rate, n = None, len(reqs)
            arr = np.zeros(n)
        else:
            rate = float(r)
            n = int(min(len(reqs), max(50, rate * args.serve_seconds)))
            arr = synth.poisson_arrivals(rate, n, seed=spec.seed + int(rate))
        served, served_res = serve_leg(gn, ix, reqs[:n], arr, budget)
        n_plain = min(n, 1000)
        plain, plain_res = plain_leg(gn, ix, reqs[:n_plain], arr[:n_plain], stream)
        # identical results: each request served in the mix against the same request on the plain path
        served["compared_with_plain"] = n_plain
        served["mismatches"] = sum(0 if same_result(a, b) else 1 for a, b in zip(served_res, plain_res))
        log(f"serving at {r} q/s: served {served['kbp_s']:.0f} kbp/s p50 {served['p50_ms']:.1f} ms "
            f"p99 {served['p99_ms']:.1f} ms; plain {plain['kbp_s']:.0f} kbp/s p50 {plain['p50_ms']:.1f} ms "
            f"p99 {plain['p99_ms']:.1f} ms; mismatches {served['mismatches']} of {n_plain}")
        out["rates"].append({"rate_qps": rate if rate is not None else "max (all at t=0)",
                             "served": served, "plain": plain})
    return out


def matches_oracle(got, exp):
    """A GPU result (gn_hit records) against the oracle's ranked alignments of the same query."""
    import numpy as np
    if len(got) != len(exp):
        return False
    for a, b in (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"), ("db_end", "de"),
                 ("score", "score"), ("rank", "rank")):
        if not np.array_equal(got[a].astype(np.int64), exp[b].astype(np.int64)):
            return False
    tiny = (np.abs(got["evalue"]) < 1e-300) & (np.abs(exp["evalue"]) < 1e-300)
    return bool((tiny | np.isclose(got["evalue"], exp["evalue"], rtol=1e-9, atol=0)).all())


def sub_leg(gn, ix, bank, queries, desc, steps, warmup, stream, dev, parity_idx, log, band_w=16, tuned=None):
    """One gn_search over a whole query set per step (device-resident queries, CUDA events around
    the steps, as the main leg), then the sampled queries parity_idx against the oracle (an index
    restricted to their seed codes, which searches them as the full one does)."""
    import oracle
    import torch
    sh = stream.cuda_stream
    qd = torch.from_numpy(queries.bases).to(f"cuda:{dev}")
    M = int(queries.start[-1])
    sp = gn.make_params(band_w=band_w)
    for _ in range(warmup):
        gn.search(ix, queries.start, qd, params=sp, stream=sh).close()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        gn.search(ix, queries.start, qd, params=sp, stream=sh).close()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    res = gn.search(ix, queries.start, qd, params=sp, stream=sh)
    got = [res.query(i).copy() for i in parity_idx]
    res.close()
    sub = queries.subset(parity_idx)
    threads = os.cpu_count() or 1
    ox = oracle.Index(bank, k=11, stride=ix.stride, restrict_to=sub, threads=threads)
    ref = ox.search(sub, oracle.Params(stride=ix.stride, band_w=band_w), threads=threads)
    mism = sum(0 if matches_oracle(g, r.ranked) else 1 for g, r in zip(got, ref))
    out = {"workload": desc, "queries": queries.n, "query_bases": M, "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "value": M / 1e3 / (ms / 1e3), "unit": UNIT, "band_w": band_w, "autotune": tuned,
           "oracle_parity": {"queries_compared": len(parity_idx), "mismatches": mism}}
    log(f"sub-leg {desc[:40]}...: {out['value']:.0f} kbp/s, {ms:.2f} ms per step, "
        f"oracle mismatches {mism} of {len(parity_idx)}")
    return out


# ----------------------------------------------------------------- arms --
def run_reference(args, dist):
    if dist.rank != 0:
        return 0
    bank, queries, desc = workload(args.workload, args.stride, 0, args.queries)
    import oracle
    threads = os.cpu_count() or 1
    ox = oracle.Index(bank, k=11, stride=args.stride, mask=args.mask)
    # size one step to about cpu_seconds / 3 of oracle time
    per_step = 8
    while True:
        sub = queries.subset(range(per_step))
        t0 = time.perf_counter()
        ox.search(sub, oracle.Params(stride=args.stride), threads=threads)
        dt = time.perf_counter() - t0
        if dt > args.cpu_seconds / 6 or per_step >= queries.n:
            break
        per_step = min(queries.n, per_step * 2)
    times, bases = [], 0
    for step in range(args.warmup + args.steps):
        lo = (step * per_step) % queries.n
        idx = [(lo + i) % queries.n for i in range(per_step)]
        sub = queries.subset(idx)
        t0 = time.perf_counter()
        ox.search(sub, oracle.Params(stride=args.stride), threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            bases += int(sub.start[-1])
    total = sum(times)
    value = bases / 1e3 / total
    sample = f"{per_step} queries per step (consecutive, wrapping), all {threads} host threads, index resident"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": desc, "stride": args.stride},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, dist):
    import numpy as np
    import torch

    import paper_1507_02987_gb300 as gn

    dev = dist.local if torch.cuda.device_count() > dist.local else 0
    torch.cuda.set_device(dev)
    gn.load()
    log = lambda *a: print(f"[rank {dist.rank}]", *a, file=sys.stderr, flush=True)

    t = time.perf_counter()
    bank, queries, desc = workload(args.workload, args.stride, dist.rank, args.queries)
    log(f"workload generated in {time.perf_counter() - t:.1f}s: {bank.n_seqs} seqs, {bank.n_bases} bases, "
        f"{queries.n} queries, {int(queries.start[-1])} query bases")
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gn.Index(bank.seq_start, bank.bases, k=11, stride=args.stride, stream=sh, mask=args.mask)
    torch.cuda.synchronize()
    t_index = time.perf_counter() - t0
    info = ix.info()
    log(f"index built in {t_index:.2f}s: {info.n_postings} postings, {info.device_bytes / 2**30:.2f} GiB")

    qd = torch.from_numpy(queries.bases).to(f"cuda:{dev}")
    qh = torch.empty(len(queries.bases), dtype=torch.uint8, pin_memory=True)
    qh.numpy()[:] = queries.bases
    qstart = queries.start
    M = int(qstart[-1])
    flags_t = gn.GN_FLAG_TIME_KERNELS

    # optional autotuner on an evenly spaced calibration sample (before any timed work)
    band_w, tuned = 16, None
    if args.autotune:
        t0 = time.perf_counter()
        cal = queries.subset(list(range(0, queries.n, max(1, queries.n // 200)))[:200])
        tp, tuning = gn.autotune(ix, cal.start, cal.bases, stream=sh)
        band_w = int(tp.band_w)
        tuned = {"band_w": band_w, **tuning, "calibration_queries": cal.n, "seconds": time.perf_counter() - t0}
        log(f"autotuned: {tuned}")
    sp = gn.make_params(band_w=band_w)
    for _ in range(args.warmup):
        gn.search(ix, qstart, qd, params=sp, stream=sh).close()
    torch.cuda.synchronize()

    # ---- timed region: device-resident queries, events on the launching stream around the K steps
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    time.sleep(0.4)
    launches0 = gn.gn_kernel_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_hits = 0
    e0.record(stream)
    for _ in range(args.steps):
        r = gn.search(ix, qstart, qd, params=sp, stream=sh)
        n_hits = r.n_queries and gn.gn_results_count(r.handle)[1]
        r.close()
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    launches = gn.gn_kernel_launch_count() - launches0
    ms_local = e0.elapsed_time(e1) / args.steps
    ms_step = dist.max(ms_local)
    bases_all = dist.sum(float(M))
    value = bases_all / 1e3 / (ms_step / 1e3)

    # ---- the same steps again with per-kernel CUDA events (each launch bracketed on its stream):
    # kernel times and work units for the rooflines (this pass is not the timed one)
    kern = {}
    phases = {}
    for _ in range(args.steps):
        r = gn.search(ix, qstart, qd, params=gn.make_params(flags=flags_t, band_w=band_w), stream=sh)
        for name, (ms, la, un) in ix.kernel_times().items():
            a = kern.setdefault(name, [0.0, 0, 0])
            a[0] += ms; a[1] += la; a[2] += un
        for name, ms in ix.phase_times().items():
            phases[name] = phases.get(name, 0.0) + ms
        r.close()
    torch.cuda.synchronize()

    # ---- end to end through the public call with pinned host queries and host results
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(args.steps):
        r = gn.search(ix, qstart, qh, params=sp, stream=sh)
        nq, nh = gn.gn_results_count(r.handle)
        d2h = nh * gn.HIT_DTYPE.itemsize
        r.close()
    torch.cuda.synchronize()
    e2e_s = dist.max((time.perf_counter() - t0) / args.steps)
    e2e = {"value": bases_all / 1e3 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": M + 8 * (queries.n + 1),
           "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s}

    # ---- plain per-query path on a sample (one gn_search per query), same GPU
    plain = None
    if args.plain_queries > 0:
        idx = list(range(0, queries.n, max(1, queries.n // args.plain_queries)))[:args.plain_queries]
        sub = queries.subset(idx)
        subs = [(np.array([0, int(sub.start[i + 1] - sub.start[i])], dtype=np.uint64),
                 torch.from_numpy(sub.bases[int(sub.start[i]):int(sub.start[i + 1])]).to(f"cuda:{dev}"))
                for i in range(sub.n)]
        for st, b in subs[:3]:
            gn.search(ix, st, b, params=sp, stream=sh).close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for st, b in subs:
            gn.search(ix, st, b, params=sp, stream=sh).close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        batched_sub = gn.search(ix, sub.start, torch.from_numpy(sub.bases).to(f"cuda:{dev}"), stream=sh)
        batched_sub.close()
        plain = {"value": int(sub.start[-1]) / 1e3 / dt, "unit": UNIT,
                 "sample": f"{sub.n} evenly spaced queries, one gn_search call per query"}

    # ---- serving: Poisson arrivals through the request loop and through the plain path
    serve = serving(args, gn, ix, bank, sh, log) if dist.rank == 0 else None

    # ---- sub-legs (rank 0, large workload only): the batched workload (10,000 queries on the mid
    # bank) and the long-query workload (40 queries of 65,536 bp - 1 Mbp on this bank and index)
    legs = None
    if dist.rank == 0 and args.workload == "large" and not args.no_sub_legs and not args.queries and not args.mask:
        import synth
        legs = {}
        lq = synth.make_queries("long", bank)
        order = sorted(range(lq.n), key=lambda i: int(lq.start[i + 1] - lq.start[i]))
        legs["long"] = sub_leg(gn, ix, bank, lq, workload_desc("long", args.stride), 3, 3, stream, dev,
                               sorted(order[:3]), log)
        bb = synth.make_bank("batched")
        bq = synth.make_queries("batched", bb)
        bix = gn.Index(bb.seq_start, bb.bases, k=11, stride=args.stride, stream=sh)
        # the batched workload's band width and kernel settings from the autotuner, on an evenly
        # spaced 200-query calibration sample, before the timed steps
        t0 = time.perf_counter()
        cal = bq.subset(list(range(0, bq.n, bq.n // 200))[:200])
        tp, tuning = gn.autotune(bix, cal.start, cal.bases, stream=sh)
        tuned = {"band_w": int(tp.band_w), **tuning, "calibration_queries": cal.n,
                 "seconds": time.perf_counter() - t0}
        log(f"batched sub-leg autotuned: {tuned}")
        pidx = list(range(0, bq.n, bq.n // 40))[:40] + [bq.n - 1]
        legs["batched"] = sub_leg(gn, bix, bb, bq, workload_desc("batched", args.stride), 5, 3, stream, dev,
                                  pidx, log, band_w=int(tp.band_w), tuned=tuned)
        if int(tp.band_w) != 16:  # the same workload at the default band, with the tuned kernel settings
            legs["batched_default_band"] = sub_leg(gn, bix, bb, bq, workload_desc("batched", args.stride), 5, 3,
                                                   stream, dev, pidx, log, band_w=16, tuned=tuned)
        bix.close()

    # ---- roofline of the dominant kernel (and of the next ones)
    peaks = measured_peaks()
    int_peaks = gn.gn_measure_int_peaks(sh)
    torch.cuda.synchronize()
    try:
        n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    except Exception:
        n_sms = None

    def roof_for(name):
        ms, la, un = kern[name]
        if name in ALU_KERNELS:
            peak = int_peaks["dpx_addmax_ops"] / 1e12 if int_peaks else None
            achieved = un * ALU_OPS_PER_UNIT / (ms / 1e3) / 1e12
            return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                    "peak_source": ("measured in this run: DPX add-max (__viaddmax_s32) throughput, 2 operations "
                                    "per instruction, all SMs") if peak else None,
                    "frac": (achieved / peak) if peak else None, "traffic": None,
                    "gcups": un / (ms / 1e3) / 1e9, "avg_launch_ms": ms / la, "launches": la}
        bpu = BYTES_PER_UNIT.get(name)
        extra = 8.0 * kern["k_bucket_group"][2] if (name == "k_bucket_fill" and "k_bucket_group" in kern) else 0.0
        achieved = (un * bpu + extra) / (ms / 1e3) / 1e9 if bpu else None
        peak = peaks.get("hbm_gbs")
        tpu = ncu_traffic(name)
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                "peak_source": "measured" if peak else None, "unit": "GB/s",
                "frac": (achieved / peak) if (achieved and peak) else None,
                "traffic": (tpu * un / la) if tpu else None,
                "algorithmic_bytes_per_launch": ((un * bpu + extra) / la) if bpu else None,
                "avg_launch_ms": ms / la, "launches": la}

    ranked = sorted(kern, key=lambda k: -kern[k][0])
    roof = roof_for(ranked[0]) if ranked else None
    roofs = [roof_for(k) for k in ranked[:4] if k in ALU_KERNELS or k in BYTES_PER_UNIT]
    kernels_out = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                       "units_per_step": v[2] / args.steps} for k, v in sorted(kern.items(), key=lambda kv: -kv[1][0])}

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1), with a parity check of that sample
    cpu = None
    parity = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        kbps, dt, sample, idx, ref, ox = oracle_run(bank, queries, args.stride, threads, args.cpu_seconds,
                                                    mask=args.mask, band_w=band_w)
        cpu = {"value": kbps, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample, "seconds": dt}
        # the same oracle on one host thread, on an evenly spaced sample of about cpu_seconds / 4
        import oracle
        one = list(range(0, queries.n, max(1, queries.n // 64)))[:64]
        sub1 = queries.subset(one)
        t0 = time.perf_counter()
        ox.search(sub1, oracle.Params(stride=args.stride, band_w=band_w), threads=1)
        dt1 = time.perf_counter() - t0
        cpu["single_thread"] = {"value": int(sub1.start[-1]) / 1e3 / dt1, "unit": UNIT, "cores": 1,
                                "sample": f"{sub1.n} evenly spaced queries, {int(sub1.start[-1])} bases",
                                "seconds": dt1}
        full = gn.search(ix, qstart, qd, params=sp, stream=sh)
        mism = 0
        for j, qi in enumerate(idx):
            got = full.query(qi)
            exp = ref[j].ranked
            same = len(got) == len(exp) and all(
                np.array_equal(got[a].astype(np.int64), exp[b].astype(np.int64))
                for a, b in (("seq", "seq"), ("q_start", "qs"), ("q_end", "qe"), ("db_start", "ds"),
                             ("db_end", "de"), ("score", "score"), ("rank", "rank")))
            same = same and np.allclose(got["evalue"], exp["evalue"], rtol=1e-9, atol=1e-300)
            mism += 0 if same else 1
        full.close()
        parity = {"queries_compared": len(idx), "mismatches": mism}

    if dist.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": desc, "bank_bases": bank.n_bases, "bank_seqs": bank.n_seqs,
                           "n_queries": queries.n, "query_bases_per_rank": M, "k": 11, "stride": args.stride,
                           "mask": args.mask, "band_w": band_w, "autotune": tuned,
                           "hits_per_step": (kern.get("k_bucket_fill") or kern.get("k_seed_gather") or [0, 0, 0])[2]
                           / max(1, args.steps),
                           "parallelism": f"replicas x{dist.world}",
                           "l2": "inputs larger than L2 (postings and hit keys are GBs per step); no flush"},
                "clocks": clk, "e2e": e2e, "gpu_launches": launches,
                "gpu_launches_per_step": launches / max(1, args.steps), "roofline": roof,
                "kernel_rooflines": roofs,
                "int_peaks_tops": {k: (v / 1e12 if k != "sms" else v) for k, v in int_peaks.items()},
                "cpu_baseline": cpu, "plain_per_query": plain, "serving": serve, "sub_legs": legs,
                "oracle_parity_on_sample": parity,
                "index_build": {"seconds": t_index, "bank_gbp_per_s": bank.n_bases / 1e9 / t_index,
                                "postings": info.n_postings, "device_gib": info.device_bytes / 2**30,
                                "includes": "host-to-device copy of the bank + pack + windows + scan + sort"},
                "phase_ms_per_step": {k: v / args.steps for k, v in phases.items()},
                "kernels": kernels_out, "alignments_per_step": n_hits,
                "kernel_timing": "per-kernel CUDA events from a second, instrumented pass of the same K steps; "
                                 "the timed pass records events only around the K steps"}
        print(json.dumps(line), flush=True)
    ix.close()
    return 0


# minimum HSP length, maximum hit distance (0: 3 x stride) and drop-off of each sweep point;
# the first is the default.  With stride 11 any two hits of a chain span >= 22 query
# bases, so lengths 12..22 select the same HSPs: 11 (single hits) is the next step down.
SWEEP_GRID = [(0, 0, 20), (11, 0, 20), (33, 0, 20), (44, 0, 20), (0, 11, 20), (0, 22, 20), (0, 66, 20),
              (0, 0, 10), (0, 0, 40)]


def run_sweep(args, dist):
    """Sensitivity sweep (the paper's minimum-HSP-length experiment, section "Results
    quality"): for each parameter point, the time per step of the whole query set and the
    planted homologs recovered, by divergence and E-value threshold."""
    import torch

    import paper_1507_02987_gb300 as gn
    from paper_1507_02987_gb300.sensitivity import recovery_table

    if dist.rank:
        return 0
    dev = dist.local if torch.cuda.device_count() > dist.local else 0
    torch.cuda.set_device(dev)
    gn.load()
    bank, queries, desc = workload(args.workload, args.stride, 0, args.queries)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ix = gn.Index(bank.seq_start, bank.bases, k=11, stride=args.stride, stream=sh, mask=args.mask)
    qd = torch.from_numpy(queries.bases).to(f"cuda:{dev}")
    M = int(queries.start[-1])
    points = []
    for min_len, dist_max, xdrop in SWEEP_GRID:
        sp = gn.make_params(max_hit_distance=dist_max, min_hsp_len=min_len, xdrop=xdrop)
        for _ in range(max(1, args.warmup)):
            gn.search(ix, queries.start, qd, params=sp, stream=sh).close()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            gn.search(ix, queries.start, qd, params=sp, stream=sh).close()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        r = gn.search(ix, queries.start, qd, params=sp, stream=sh)
        res = r.all()
        r.close()
        k = ix.k
        points.append({"min_hsp_len": min_len or 2 * k, "max_hit_distance": dist_max or 3 * args.stride,
                       "xdrop": xdrop, "ms_per_step": ms, "value": M / 1e3 / (ms / 1e3),
                       "alignments": int(sum(len(a) for a in res)),
                       "recovery": recovery_table(queries.meta, res)})
        print(f"[sweep] {points[-1]['min_hsp_len']:3d} {points[-1]['max_hit_distance']:3d} {xdrop:3d}: "
              f"{ms:8.2f} ms, found {points[-1]['recovery']['found']} of {points[-1]['recovery']['planted']}",
              file=sys.stderr, flush=True)
    ix.close()
    print(json.dumps({"mode": "sensitivity_sweep", "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": desc, "mask": args.mask, "band_w": 16},
                      "data": "synthetic", "sweep": points}), flush=True)
    return 0


def main():
    args = parse_args()
    dist = Dist()
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        if args.sweep:
            return run_sweep(args, dist)
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
