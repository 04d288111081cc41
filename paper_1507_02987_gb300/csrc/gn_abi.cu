// gn_abi.cu - the extern "C" boundary: argument checking, error reporting,
// handle ownership, and the serving loop (continuous batching).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "gn_internal.cuh"

namespace gn {
static thread_local std::string g_last_error;

void set_error(gn_status st, const std::string &msg) {
    (void)st;
    g_last_error = msg;
}

template <class F>
static gn_status guarded(F &&f) {
    try {
        f();
        g_last_error.clear();
        return GN_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return GN_ENOMEM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return GN_EINTERNAL;
    }
}

static void resolve(const gn_index *ix, const gn_scoring *sc, const gn_params *pp, SearchOptions &o) {
    gn_default_params(&o.sc, &o.p);
    if (sc) o.sc = *sc;
    if (pp) o.p = *pp;
    if (o.p.max_hit_distance == 0) o.p.max_hit_distance = 3u * (uint32_t)ix->t;
    if (o.p.min_hsp_len == 0) o.p.min_hsp_len = 2u * (uint32_t)ix->k;
    GN_REQUIRE(o.p.xdrop >= 0, GN_EINVAL, "xdrop must be >= 0");
    GN_REQUIRE(o.p.band_w <= 16384, GN_EINVAL, "band_w must be <= 16384");
    GN_REQUIRE(o.p.max_hit_distance < 65536, GN_EINVAL, "max_hit_distance must be < 65536");
    GN_REQUIRE(o.sc.gap_extend <= 0 && o.sc.gap_open <= 0, GN_EINVAL, "gap scores must be <= 0");
    GN_REQUIRE(o.sc.match > 0 && o.sc.mismatch < 0, GN_EINVAL, "match must be > 0 and mismatch < 0");
    GN_REQUIRE(o.sc.K > 0 && o.sc.lambda > 0, GN_EINVAL, "lambda and K must be > 0");
}

static void check_queries(const gn_queries *q, uint64_t max_len = MAX_QUERY_LEN) {
    GN_REQUIRE(q && q->start, GN_EINVAL, "queries and queries.start are required");
    GN_REQUIRE(q->n <= MAX_QUERIES, GN_ETOOBIG, "at most 65,536 queries per call");
    GN_REQUIRE(q->start[0] == 0, GN_EINVAL, "queries.start[0] must be 0");
    for (uint32_t i = 0; i < q->n; ++i) {
        GN_REQUIRE(q->start[i + 1] >= q->start[i], GN_EINVAL, "queries.start must be non-decreasing");
        GN_REQUIRE(q->start[i + 1] - q->start[i] <= max_len, GN_ETOOBIG,
                   max_len == MAX_QUERY_LEN ? "a query holds 65,536 bases or more" : "a query holds 2^24 bases or more");
    }
    GN_REQUIRE(q->start[q->n] == 0 || q->bases, GN_EINVAL, "queries.bases is required");
}

// ------------------------------------------------------------ serving --
constexpr uint64_t FOOTPRINT_UNKNOWN = ~0ull;

// A submitted query.  Its footprint is unknown until a worker has counted its seed hits
// on the device (`counting` while one does); a request whose count failed carries the
// error and fails when it reaches the head of the queue.
struct Request {
    uint64_t ticket;
    std::string bases;
    uint64_t footprint = FOOTPRINT_UNKNOWN;
    bool counting = false;
    gn_status status = GN_OK;
    std::string err;
};

}  // namespace gn

struct gn_server {
    const gn_index *ix = nullptr;
    gn::SearchOptions opt;
    uint64_t budget = 0;
    uint64_t in_use = 0;
    bool stopping = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<gn::Request> queue;
    std::map<uint64_t, gn_results *> done;
    std::map<uint64_t, std::pair<gn_status, std::string>> failed;
    uint64_t next_ticket = 1;
    uint64_t count_from = 1;  // requests with smaller tickets are counted, or being counted
    std::vector<std::thread> workers;
    int device = 0;
    gn_serve_stats stats{};
    uint64_t running = 0;  // micro-batches on the device now
};

namespace gn {
// Device bytes one batch needs besides its queries' own footprints (initial HSP and spill
// buffers, counters, scan scratch).
constexpr uint64_t BATCH_FIXED_BYTES = 16ull << 20;

// Admission footprint of one query: its exact seed-hit count times the bytes a chunk
// budgets per hit, its per-offset arrays, its smallest set of hit buckets (two of 1,024
// entries), and the alignment records of its selected HSPs.
static uint64_t footprint_of(const gn_server *sv, uint64_t hits, uint64_t len) {
    const uint64_t n_sel = sv->opt.p.max_alignments ? sv->opt.p.max_alignments : 4096;
    return hits * HIT_BYTES + len * 64 + 2 * 1024 * 8 + n_sel * (64 + 16 * (2ull * sv->opt.p.band_w + 2));
}

// Requests a worker counts in one launch.
constexpr size_t COUNT_MAX_REQUESTS = 4096;
constexpr uint64_t COUNT_MAX_BASES = 16ull << 20;

// Device buffer that only grows (one per worker and purpose), stream-ordered on the worker's
// stream: growing it waits for nothing the other workers run (a plain free would wait for the
// whole device).
struct GrowBuf {
    cudaStream_t s = nullptr;
    void *p = nullptr;
    size_t cap = 0;
    void *get(size_t bytes) {
        if (bytes > cap) {
            if (p) GN_CUDA(cudaFreeAsync(p, s));
            p = nullptr;
            cap = 0;
            const size_t want = std::max<size_t>(bytes, 1 << 20);
            GN_CUDA(cudaMallocAsync(&p, want, s));
            cap = want;
        }
        return p;
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        cap = 0;
    }
};

static void serve_worker(gn_server *sv) {
    cudaSetDevice(sv->device);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    GrowBuf dbases{s}, dstart{s}, dhits{s};
    auto first_uncounted = [&]() -> size_t {  // position of the first request not yet claimed for counting
        auto it = std::lower_bound(sv->queue.begin(), sv->queue.end(), sv->count_from,
                                   [](const Request &r, uint64_t t) { return r.ticket < t; });
        return (size_t)(it - sv->queue.begin());
    };
    for (;;) {
        std::vector<Request> batch;
        std::vector<Request *> tocount;
        uint64_t taken = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                if (sv->queue.empty()) return sv->stopping;
                if (first_uncounted() < sv->queue.size()) return true;
                const Request &f = sv->queue.front();
                if (f.footprint == FOOTPRINT_UNKNOWN) return false;
                return f.status != GN_OK || f.footprint + BATCH_FIXED_BYTES > sv->budget ||
                       sv->in_use + BATCH_FIXED_BYTES + f.footprint <= sv->budget;
            });
            if (sv->queue.empty()) break;
            const size_t k = first_uncounted();
            const uint64_t rest = sv->budget - BATCH_FIXED_BYTES;
            if (k == 0 && sv->running == 0 && sv->in_use == 0 &&
                footprint_of(sv, 0, sv->queue.front().bases.size()) < rest) {
                // nothing runs: the head request runs at once, alone, with the whole budget (its hit
                // storage capped to what the budget leaves), without waiting for its count
                taken = sv->budget;
                sv->count_from = sv->queue.front().ticket + 1;
                batch.push_back(std::move(sv->queue.front()));
                sv->queue.pop_front();
                sv->in_use += taken;
                sv->stats.batches += 1;
                sv->stats.requests += 1;
                sv->stats.max_batch = std::max<uint64_t>(sv->stats.max_batch, 1);
                sv->running += 1;
                sv->stats.max_concurrent = std::max(sv->stats.max_concurrent, sv->running);
                sv->stats.peak_in_use = std::max(sv->stats.peak_in_use, sv->in_use);
            } else if (k < sv->queue.size()) {
                // claim the next arrivals for counting (in arrival order)
                uint64_t nb = 0;
                for (size_t i = k; i < sv->queue.size() && tocount.size() < COUNT_MAX_REQUESTS && nb < COUNT_MAX_BASES;
                     ++i) {
                    Request &r = sv->queue[i];
                    r.counting = true;
                    tocount.push_back(&r);
                    nb += r.bases.size();
                }
                sv->count_from = tocount.back()->ticket + 1;
            } else {
                Request &f = sv->queue.front();
                if (f.status != GN_OK || f.footprint + BATCH_FIXED_BYTES > sv->budget) {
                    // a request that cannot run: its count failed, or it alone exceeds the budget
                    if (f.status != GN_OK) sv->failed[f.ticket] = {f.status, f.err};
                    else sv->failed[f.ticket] = {GN_ETOOBIG, "the query alone exceeds the server's memory budget"};
                    sv->queue.pop_front();
                    lk.unlock();
                    sv->cv_done.notify_all();
                    continue;
                }
                // admit counted arrivals in order while they fit the memory budget (continuous batching)
                taken = BATCH_FIXED_BYTES;
                while (!sv->queue.empty() && batch.size() < MAX_QUERIES) {
                    const Request &r = sv->queue.front();
                    if (r.footprint == FOOTPRINT_UNKNOWN || r.status != GN_OK ||
                        sv->in_use + taken + r.footprint > sv->budget)
                        break;
                    taken += r.footprint;
                    batch.push_back(std::move(sv->queue.front()));
                    sv->queue.pop_front();
                }
                sv->in_use += taken;
                sv->stats.batches += 1;
                sv->stats.requests += batch.size();
                sv->stats.max_batch = std::max<uint64_t>(sv->stats.max_batch, batch.size());
                sv->running += 1;
                sv->stats.max_concurrent = std::max(sv->stats.max_concurrent, sv->running);
                sv->stats.peak_in_use = std::max(sv->stats.peak_in_use, sv->in_use);
            }
        }
        if (!tocount.empty()) {
            // seed hits of the claimed requests, counted on the device (the requests stay in the
            // queue: only the head is ever removed, and not while a request is being counted)
            const uint32_t n = (uint32_t)tocount.size();
            std::vector<uint64_t> start(n + 1, 0);
            for (uint32_t i = 0; i < n; ++i) start[i + 1] = start[i] + tocount[i]->bases.size();
            std::vector<unsigned long long> hits(n, 0);
            gn_status st = guarded([&] {
                std::string host;
                host.reserve(start[n]);
                for (auto *r : tocount) host += r->bases;
                uint8_t *b = static_cast<uint8_t *>(dbases.get(std::max<uint64_t>(start[n], 1)));
                uint64_t *st_d = static_cast<uint64_t *>(dstart.get(8 * (n + 1)));
                unsigned long long *h_d = static_cast<unsigned long long *>(dhits.get(8 * n));
                if (start[n]) GN_CUDA(cudaMemcpyAsync(b, host.data(), start[n], cudaMemcpyHostToDevice, s));
                GN_CUDA(cudaMemcpyAsync(st_d, start.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s));
                count_request_hits(sv->ix, b, st_d, n, h_d, s);
                GN_CUDA(cudaMemcpyAsync(hits.data(), h_d, 8 * n, cudaMemcpyDeviceToHost, s));
                GN_CUDA(cudaStreamSynchronize(s));
            });
            const std::string err = st != GN_OK ? g_last_error : std::string();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                for (uint32_t i = 0; i < n; ++i) {
                    Request *r = tocount[i];
                    r->counting = false;
                    r->footprint = footprint_of(sv, hits[i], r->bases.size());
                    if (st != GN_OK) { r->status = st; r->err = err; }
                }
            }
            sv->cv_work.notify_all();
            continue;
        }
        std::vector<uint64_t> qstart(batch.size() + 1, 0);
        for (size_t i = 0; i < batch.size(); ++i) qstart[i + 1] = qstart[i] + batch[i].bases.size();
        std::string err;
        gn_results all;
        gn_status st = guarded([&] {
            uint64_t M = qstart.back();
            uint8_t *b = static_cast<uint8_t *>(dbases.get(std::max<uint64_t>(M, 1)));
            std::string host;
            host.reserve(M);
            for (auto &r : batch) host += r.bases;
            if (M) GN_CUDA(cudaMemcpyAsync(b, host.data(), M, cudaMemcpyHostToDevice, s));
            SearchOptions o = sv->opt;
            // the hit storage stays inside what was admitted (a lone request admitted before its
            // count: the budget less its other arrays)
            o.mem_cap = taken - BATCH_FIXED_BYTES;
            if (batch.size() == 1 && batch[0].footprint == FOOTPRINT_UNKNOWN) {
                o.mem_cap -= footprint_of(sv, 0, batch[0].bases.size());
                o.max_hit_bytes = o.mem_cap;  // as admission would: GN_ETOOBIG if it cannot fit even alone
            }
            search(const_cast<gn_index *>(sv->ix), b, qstart, o, s, &all);
        });
        if (st != GN_OK) err = g_last_error;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (size_t i = 0; i < batch.size(); ++i) {
                if (st != GN_OK) {
                    sv->failed[batch[i].ticket] = {st, err};
                    continue;
                }
                gn_results *r = new gn_results();
                r->n_queries = 1;
                r->qoff = {0, all.qoff[i + 1] - all.qoff[i]};
                r->hits.assign(all.hits.begin() + all.qoff[i], all.hits.begin() + all.qoff[i + 1]);
                for (auto &h : r->hits) h.query = 0;
                sv->done[batch[i].ticket] = r;
            }
            sv->in_use -= taken;
            sv->running -= 1;
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    dbases.release();
    dstart.release();
    dhits.release();
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
}
}  // namespace gn

using namespace gn;

extern "C" {

gn_status gn_default_params(gn_scoring *sc, gn_params *p) {
    if (sc) {
        sc->match = 1;
        sc->mismatch = -3;
        sc->gap_open = -5;
        sc->gap_extend = -2;
        sc->lambda = 1.3740631;
        sc->K = 0.711;
    }
    if (p) {
        p->max_hit_distance = 0;
        p->min_hsp_len = 0;
        p->xdrop = 20;
        p->max_alignments = 100;
        p->band_w = 16;
        p->max_evalue = INFINITY;
        p->flags = 0;
    }
    return GN_OK;
}

gn_status gn_index_build(const gn_bank *db, int k, int stride, void *cuda_stream, gn_index **out) {
    if (!out) { g_last_error = "out is required"; return GN_EINVAL; }
    *out = nullptr;
    gn_index *ix = new (std::nothrow) gn_index();
    if (!ix) { g_last_error = "host allocation failed"; return GN_ENOMEM; }
    gn_status st = guarded([&] { index_build(db, k, stride, (cudaStream_t)cuda_stream, ix); });
    if (st != GN_OK) {
        std::string msg = g_last_error;
        index_free(ix);
        delete ix;
        g_last_error = msg;
        return st;
    }
    *out = ix;
    return GN_OK;
}

gn_status gn_index_build_masked(const gn_bank *db, const char *mask, int stride, void *cuda_stream, gn_index **out) {
    if (!out) { g_last_error = "out is required"; return GN_EINVAL; }
    *out = nullptr;
    gn_index *ix = new (std::nothrow) gn_index();
    if (!ix) { g_last_error = "host allocation failed"; return GN_ENOMEM; }
    gn_status st = guarded([&] { index_build_masked(db, mask, stride, (cudaStream_t)cuda_stream, ix); });
    if (st != GN_OK) {
        std::string msg = g_last_error;
        index_free(ix);
        delete ix;
        g_last_error = msg;
        return st;
    }
    *out = ix;
    return GN_OK;
}

gn_status gn_index_set_tuning(gn_index *ix, const gn_tuning *t) {
    if (!ix || !t) { g_last_error = "index and tuning are required"; return GN_EINVAL; }
    if (t->fill_threads != 0 && t->fill_threads != 256 && t->fill_threads != 512) {
        g_last_error = "fill_threads is 0, 256 or 512";
        return GN_EINVAL;
    }
    if (t->sw_lanes != 0 && t->sw_lanes != 8 && t->sw_lanes != 16 && t->sw_lanes != 32) {
        g_last_error = "sw_lanes is 0, 8, 16 or 32";
        return GN_EINVAL;
    }
    ix->tuning = *t;
    return GN_OK;
}

gn_status gn_index_get_tuning(const gn_index *ix, gn_tuning *t) {
    if (!ix || !t) { g_last_error = "index and tuning are required"; return GN_EINVAL; }
    *t = ix->tuning;
    return GN_OK;
}

gn_status gn_autotune(gn_index *ix, const gn_queries *q, const gn_scoring *sc, gn_params *p, uint32_t what,
                      void *cuda_stream, gn_tuning *tuning) {
    if (!ix || !q || !p) { g_last_error = "index, sample and params are required"; return GN_EINVAL; }
    return guarded([&] {
        check_queries(q);
        cudaStream_t s = (cudaStream_t)cuda_stream;
        std::vector<uint64_t> qstart(q->start, q->start + q->n + 1);
        const uint64_t M = qstart[q->n];
        DeviceArena arena(s);
        const uint8_t *qd = reinterpret_cast<const uint8_t *>(q->bases);
        if (q->bases_mem == GN_MEM_HOST && M > 0) {
            uint8_t *tmp = arena.alloc_n<uint8_t>(M);
            GN_CUDA(cudaMemcpyAsync(tmp, q->bases, M, cudaMemcpyHostToDevice, s));
            qd = tmp;
        }
        auto run = [&](const gn_params &pp, gn_results &res) {
            SearchOptions o;
            gn_params p2 = pp;
            p2.flags &= ~(GN_FLAG_KEEP_STAGES | GN_FLAG_KEEP_HITS | GN_FLAG_BOTH_STRANDS | GN_FLAG_TIME_KERNELS);
            resolve(ix, sc, &p2, o);
            search(ix, qd, qstart, o, s, &res);
        };
        auto total = [](const gn_results &a) {
            double t = 0.0;
            for (const gn_hit &h : a.hits) t += (double)h.score;
            return t;
        };
        if (what & GN_TUNE_BAND) {
            // the smallest band that a band twice as wide improves by at most 0.5 % of the sample's total
            // alignment score (a wider band recovers alignments whose indels drift off the seed diagonal)
            const uint32_t ws[] = {16, 32, 64, 128};
            gn_params pp = *p;
            uint32_t chosen = 128;
            gn_results prev;
            pp.band_w = ws[0];
            run(pp, prev);
            for (int i = 0; i + 1 < 4; ++i) {
                gn_results next;
                pp.band_w = ws[i + 1];
                run(pp, next);
                const double a = total(prev), b = total(next);
                if (b - a <= 0.005 * std::max(a, 1.0)) { chosen = ws[i]; break; }
                prev = std::move(next);
            }
            p->band_w = chosen;
        }
        if (what & GN_TUNE_KERNELS) {
            // fastest of a few result-invariant settings, by CUDA-event time on the caller's stream
            const gn_tuning saved = ix->tuning;
            gn_tuning best = saved;  // the library's defaults where unset, so that the result is explicit
            if (!best.tile_hits) best.tile_hits = 50000;
            if (!best.fill_threads) best.fill_threads = 512;
            if (!best.bucket_target) best.bucket_target = 4096;
            if (!best.sw_lanes) best.sw_lanes = 8;
            if (!best.sw_wave_rows) best.sw_wave_rows = 512;
            float best_ms = 0.f;
            bool have = false;
            cudaEvent_t e0, e1;
            GN_CUDA(cudaEventCreate(&e0));
            GN_CUDA(cudaEventCreate(&e1));
            auto time_of = [&](const gn_tuning &cand) {
                ix->tuning = cand;
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {  // the first run warms pools and caches
                    gn_results r;
                    GN_CUDA(cudaEventRecord(e0, s));
                    run(*p, r);
                    GN_CUDA(cudaEventRecord(e1, s));
                    GN_CUDA(cudaEventSynchronize(e1));
                    GN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                }
                if (!have || ms < best_ms) { best = cand; best_ms = ms; have = true; }
            };
            // one group of settings after the other, each from the best so far
            for (uint32_t th : {512u, 256u})
                for (uint32_t hits : {25000u, 50000u, 100000u}) {
                    gn_tuning cand = best;
                    cand.fill_threads = th;
                    cand.tile_hits = hits;
                    time_of(cand);
                }
            {
                const gn_tuning base = best;
                for (uint32_t bt : {2048u, 4096u, 8192u}) {
                    gn_tuning cand = base;
                    cand.bucket_target = bt;
                    time_of(cand);
                }
            }
            {
                const gn_tuning base = best;
                for (uint32_t lanes : {8u, 16u, 32u})
                    for (uint32_t rows : {256u, 512u, 1024u}) {
                        gn_tuning cand = base;
                        cand.sw_lanes = lanes;
                        cand.sw_wave_rows = rows;
                        time_of(cand);
                    }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ix->tuning = best;
        }
        if (tuning) *tuning = ix->tuning;
        arena.release();
    });
}

gn_status gn_index_save(const gn_index *ix, const char *path) {
    if (!ix) { g_last_error = "index is required"; return GN_EINVAL; }
    return guarded([&] { index_save(ix, path); });
}

gn_status gn_index_load(const char *path, gn_index **out) {
    if (!out) { g_last_error = "out is required"; return GN_EINVAL; }
    *out = nullptr;
    gn_index *ix = new (std::nothrow) gn_index();
    if (!ix) { g_last_error = "host allocation failed"; return GN_ENOMEM; }
    gn_status st = guarded([&] { index_load(path, ix); });
    if (st != GN_OK) {
        std::string msg = g_last_error;
        index_free(ix);
        delete ix;
        g_last_error = msg;
        return st;
    }
    *out = ix;
    return GN_OK;
}

void gn_index_free(gn_index *ix) {
    if (!ix) return;
    index_free(ix);
    delete ix;
}

gn_status gn_index_get_info(const gn_index *ix, gn_index_info *info) {
    if (!ix || !info) { g_last_error = "index and info are required"; return GN_EINVAL; }
    info->k = ix->k;
    info->stride = ix->t;
    info->n_seqs = ix->n_seqs;
    info->n_bases = ix->n_bases;
    info->n_postings = ix->n_postings;
    info->device_bytes = ix->device_bytes;
    return GN_OK;
}

gn_status gn_index_export(const gn_index *ix, uint64_t *bucket_start, uint32_t *post_seq, uint32_t *post_pos) {
    if (!ix) { g_last_error = "index is required"; return GN_EINVAL; }
    return guarded([&] { index_export(ix, bucket_start, post_seq, post_pos); });
}

gn_status gn_search(const gn_index *ix, const gn_queries *q, const gn_scoring *sc, const gn_params *p,
                    void *cuda_stream, gn_results **out) {
    if (!out) { g_last_error = "out is required"; return GN_EINVAL; }
    *out = nullptr;
    if (!ix) { g_last_error = "index is required"; return GN_EINVAL; }
    gn_results *res = new (std::nothrow) gn_results();
    if (!res) { g_last_error = "host allocation failed"; return GN_ENOMEM; }
    gn_status st = guarded([&] {
        check_queries(q, MAX_LONG_QUERY_LEN);
        SearchOptions o;
        resolve(ix, sc, p, o);
        int dev = 0;
        GN_CUDA(cudaGetDevice(&dev));
        GN_REQUIRE(dev == ix->device, GN_EINVAL, "the current device is not the index's device");
        cudaStream_t s = (cudaStream_t)cuda_stream;
        std::vector<uint64_t> qstart(q->start, q->start + q->n + 1);
        const uint64_t M = qstart[q->n];
        const uint8_t *qd = reinterpret_cast<const uint8_t *>(q->bases);
        DeviceArena arena(s);
        if (q->bases_mem == GN_MEM_HOST && M > 0) {
            uint8_t *tmp = arena.alloc_n<uint8_t>(M);
            GN_CUDA(cudaMemcpyAsync(tmp, q->bases, M, cudaMemcpyHostToDevice, s));
            qd = tmp;
        }
        if (o.p.flags & GN_FLAG_BOTH_STRANDS) {
            GN_REQUIRE(2ull * q->n <= MAX_QUERIES, GN_ETOOBIG, "more than 32,768 queries with both strands");
            std::vector<uint64_t> qstart2;
            both_strands(qd, qstart, arena, s, &qd, qstart2);
            qstart.swap(qstart2);
        }
        search(const_cast<gn_index *>(ix), qd, qstart, o, s, res);
        arena.release();
    });
    if (st != GN_OK) {
        delete res;
        return st;
    }
    *out = res;
    return GN_OK;
}

void gn_results_free(gn_results *r) { delete r; }

gn_status gn_results_get(const gn_results *r, uint32_t query, const gn_hit **hits, uint32_t *n) {
    if (!r || !hits || !n) { g_last_error = "results, hits and n are required"; return GN_EINVAL; }
    if (query >= r->n_queries) { g_last_error = "query index out of range"; return GN_EINVAL; }
    *n = (uint32_t)(r->qoff[query + 1] - r->qoff[query]);
    *hits = *n ? r->hits.data() + r->qoff[query] : nullptr;
    return GN_OK;
}

gn_status gn_results_count(const gn_results *r, uint32_t *nq, uint64_t *nh) {
    if (!r) { g_last_error = "results are required"; return GN_EINVAL; }
    if (nq) *nq = r->n_queries;
    if (nh) *nh = r->hits.size();
    return GN_OK;
}

gn_status gn_results_stage(const gn_results *r, gn_stage stage, const void **data, uint64_t *n) {
    if (!r || !data || !n) { g_last_error = "results, data and n are required"; return GN_EINVAL; }
    if (!r->has_stages && stage != GN_STAGE_HITS) { g_last_error = "search ran without GN_FLAG_KEEP_STAGES"; return GN_EINVAL; }
    switch (stage) {
    case GN_STAGE_HSP: *data = r->st_hsp.data(); *n = r->st_hsp.size(); break;
    case GN_STAGE_EXT: *data = r->st_ext.data(); *n = r->st_ext.size(); break;
    case GN_STAGE_MERGED: *data = r->st_merged.data(); *n = r->st_merged.size(); break;
    case GN_STAGE_SELECTED: *data = r->st_sel.data(); *n = r->st_sel.size(); break;
    case GN_STAGE_ALIGNED: *data = r->st_aln.data(); *n = r->st_aln.size(); break;
    case GN_STAGE_HITS: *data = r->st_hits.data(); *n = r->st_hits.size() / 4; break;
    case GN_STAGE_HIT_COUNTS: *data = r->st_hit_counts.data(); *n = r->st_hit_counts.size(); break;
    default: g_last_error = "unknown stage"; return GN_EINVAL;
    }
    return GN_OK;
}

int gn_last_phase_times(const gn_index *ix, const char **names, float *ms, int cap) {
    if (!ix) return 0;
    std::lock_guard<std::mutex> lk(const_cast<gn_index *>(ix)->phase_mu);
    int n = 0;
    for (auto &ph : ix->last_phases) {
        if (n >= cap) break;
        if (names) names[n] = ph.first;
        if (ms) ms[n] = ph.second;
        ++n;
    }
    return n;
}

int gn_last_kernel_times(const gn_index *ix, const char **names, double *ms, uint32_t *launches, uint64_t *units,
                         int cap) {
    if (!ix) return 0;
    std::lock_guard<std::mutex> lk(const_cast<gn_index *>(ix)->phase_mu);
    int n = 0;
    for (auto &k : ix->last_kernels) {
        if (n >= cap) break;
        if (names) names[n] = k.name;
        if (ms) ms[n] = k.ms;
        if (launches) launches[n] = k.launches;
        if (units) units[n] = k.units;
        ++n;
    }
    return n;
}

uint64_t gn_kernel_launch_count(void) { return (uint64_t)launch_count(); }

gn_status gn_serve_start(const gn_index *ix, const gn_scoring *sc, const gn_params *p, uint64_t mem_budget,
                         gn_server **out) {
    if (!out || !ix) { g_last_error = "index and out are required"; return GN_EINVAL; }
    *out = nullptr;
    gn_server *sv = new (std::nothrow) gn_server();
    if (!sv) { g_last_error = "host allocation failed"; return GN_ENOMEM; }
    gn_status st = guarded([&] {
        resolve(ix, sc, p, sv->opt);
        sv->opt.p.flags &= ~(GN_FLAG_KEEP_STAGES | GN_FLAG_KEEP_HITS | GN_FLAG_BOTH_STRANDS);
        GN_REQUIRE(mem_budget > BATCH_FIXED_BYTES, GN_EINVAL, "mem_budget must exceed 16 MiB");
        sv->ix = ix;
        sv->budget = mem_budget;
        sv->device = ix->device;
        GN_CUDA(cudaSetDevice(ix->device));
        for (int w = 0; w < 3; ++w) sv->workers.emplace_back(serve_worker, sv);
    });
    if (st != GN_OK) { delete sv; return st; }
    *out = sv;
    return GN_OK;
}

gn_status gn_serve_submit(gn_server *sv, const char *bases, uint32_t len, uint64_t *ticket) {
    if (!sv || !ticket || (len && !bases)) { g_last_error = "server, bases and ticket are required"; return GN_EINVAL; }
    if (len > MAX_QUERY_LEN) { g_last_error = "a query holds 65,536 bases or more"; return GN_ETOOBIG; }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) { g_last_error = "server is stopping"; return GN_EBUSY; }
        Request r;
        r.ticket = sv->next_ticket++;
        r.bases.assign(bases ? bases : "", len);
        *ticket = r.ticket;
        sv->queue.push_back(std::move(r));
    }
    sv->cv_work.notify_one();
    g_last_error.clear();
    return GN_OK;
}

gn_status gn_serve_poll(gn_server *sv, uint64_t ticket, uint32_t timeout_ms, gn_results **out) {
    if (!sv || !out) { g_last_error = "server and out are required"; return GN_EINVAL; }
    *out = nullptr;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] { return sv->done.count(ticket) || sv->failed.count(ticket); };
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        g_last_error = "not done yet";
        return GN_ETIMEOUT;
    }
    auto f = sv->failed.find(ticket);
    if (f != sv->failed.end()) {
        const gn_status st = f->second.first;
        g_last_error = f->second.second;
        sv->failed.erase(f);
        return st;
    }
    auto it = sv->done.find(ticket);
    *out = it->second;
    sv->done.erase(it);
    g_last_error.clear();
    return GN_OK;
}

gn_status gn_serve_poll_any(gn_server *sv, uint32_t timeout_ms, uint64_t *ticket, gn_results **out) {
    if (!sv || !out || !ticket) { g_last_error = "server, ticket and out are required"; return GN_EINVAL; }
    *out = nullptr;
    *ticket = 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] { return !sv->done.empty() || !sv->failed.empty(); };
    if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        g_last_error = "nothing done yet";
        return GN_ETIMEOUT;
    }
    // the oldest finished ticket first
    const bool take_failed = sv->done.empty() ||
                             (!sv->failed.empty() && sv->failed.begin()->first < sv->done.begin()->first);
    if (take_failed) {
        auto f = sv->failed.begin();
        *ticket = f->first;
        const gn_status st = f->second.first;
        g_last_error = f->second.second;
        sv->failed.erase(f);
        return st;
    }
    auto it = sv->done.begin();
    *ticket = it->first;
    *out = it->second;
    sv->done.erase(it);
    g_last_error.clear();
    return GN_OK;
}

gn_status gn_serve_get_stats(gn_server *sv, gn_serve_stats *out) {
    if (!sv || !out) { g_last_error = "server and out are required"; return GN_EINVAL; }
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->in_use = sv->in_use;
    out->queued = sv->queue.size();
    return GN_OK;
}

gn_status gn_serve_stop(gn_server *sv) {
    if (!sv) return GN_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (auto &kv : sv->done) delete kv.second;
    delete sv;
    return GN_OK;
}

gn_status gn_align_hsps_static(const gn_index *ix, const char *query_bases, const uint64_t *query_start,
                               uint32_t n_queries, const gn_hsp *hsps, uint32_t n_hsps, const gn_scoring *scoring,
                               uint32_t band_w, gn_hit *out, void *cuda_stream) {
    return guarded([&] {
        align_hsps_static(ix, query_bases, query_start, n_queries, hsps, n_hsps, scoring, band_w, out,
                          (cudaStream_t)cuda_stream);
    });
}

gn_status gn_measure_int_peaks(gn_int_peaks *out, void *cuda_stream) {
    return guarded([&] { measure_int_peaks(out, (cudaStream_t)cuda_stream); });
}

void gn_debug_fail_alloc(uint64_t nth) { debug_fail_alloc(nth); }

gn_status gn_debug_scan(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t wait_cycles, int drop_first,
                        void *cuda_stream) {
    return guarded([&] {
        GN_REQUIRE(out && (n == 0 || in), GN_EINVAL, "in and out are required");
        const long long budget = wait_cycles ? (long long)std::min<uint64_t>(wait_cycles, 1ull << 40) : (1ll << 31);
        const bool ran_out = debug_scan(in, out, n, budget, drop_first ? 1 : 0, (cudaStream_t)cuda_stream);
        GN_REQUIRE(!ran_out, GN_ETIMEOUT, "a device-side wait ran out (scan look-back)");
    });
}
gn_status gn_debug_sort(uint64_t *keys, uint32_t *vals, uint64_t n, int bit_lo, int bit_hi, uint64_t wait_cycles,
                        int drop_first, int three_kernel, void *cuda_stream) {
    return guarded([&] {
        GN_REQUIRE(n == 0 || keys, GN_EINVAL, "keys are required");
        GN_REQUIRE(bit_lo >= 0 && bit_hi <= 64 && bit_lo <= bit_hi, GN_EINVAL, "bits must satisfy 0 <= bit_lo <= bit_hi <= 64");
        GN_REQUIRE(n < (1ull << 32), GN_ETOOBIG, "at most 2^32 - 1 keys");
        const long long budget = wait_cycles ? (long long)std::min<uint64_t>(wait_cycles, 1ull << 40) : (1ll << 31);
        const bool ran_out = debug_sort(keys, vals, n, bit_lo, bit_hi, budget, drop_first ? 1 : 0, three_kernel != 0,
                                        (cudaStream_t)cuda_stream);
        GN_REQUIRE(!ran_out, GN_ETIMEOUT, "a device-side wait ran out (sort look-back)");
    });
}
uint64_t gn_debug_alloc_count(void) { return debug_alloc_count(); }
int64_t gn_debug_live_allocs(void) { return debug_live_allocs(); }

const char *gn_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
