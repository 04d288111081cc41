// gn_noalloc.cu - gn_align_hsps_static: banded Smith-Waterman of caller-given
// HSPs with no device allocation at all.  Some callers cannot call cudaMalloc
// (or a stream-ordered allocator) on their path: code whose device memory is
// owned by another allocator that must stay the only one, code running close
// to a hard memory limit that cannot risk an allocation failure in the middle
// of a job, or latency-critical loops that cannot afford an allocation call.
// This variant keeps its scratch in one file-scope device array instead.
#include <cstddef>
#include <mutex>

#include "gn_internal.cuh"

namespace gn {
namespace {

// Scratch shared by every call: a small header (task counter, status word)
// followed by one row strip per warp.  A strip holds the previous DP row of
// one band of up to kStaticMaxBand diagonals.
constexpr int kStaticWarps = 512;
constexpr int kStaticMaxBand = 1024;
constexpr int kStaticSlot = kStaticMaxBand + 1;

struct StaticCell {
    int32_t H, E;
    uint32_t SH, SE;
};

struct StaticScratch {
    uint32_t next_task;
    uint32_t status;
    uint32_t pad[62];
    StaticCell strips[kStaticWarps * kStaticSlot];
};

static __device__ __align__(256) StaticScratch g_static_scratch;

constexpr uint32_t kErrTooWide = 1u;
constexpr uint32_t kErrBadRecord = 2u;
constexpr int32_t kNeg = -(1 << 29);
constexpr int32_t kXNeg = -(1 << 30);

__device__ __forceinline__ uint32_t ascii_code(uint8_t b) {
    uint32_t c = b & 0xDFu;
    if (c == 'A') return 0u;
    if (c == 'C') return 1u;
    if (c == 'G') return 2u;
    if (c == 'T' || c == 'U') return 3u;
    return 4u;  // non-base
}

__device__ __forceinline__ int32_t pair_score(uint32_t a, uint32_t b, int32_t match, int32_t mismatch) {
    return (a < 4u && a == b) ? match : mismatch;
}

__device__ __forceinline__ void scan_max_later_wins(int32_t &v, uint32_t &s, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t ov = __shfl_up_sync(0xffffffffu, v, o);
        uint32_t os = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o && ov > v) { v = ov; s = os; }
    }
}

// One warp per HSP (taken from the shared task counter); the warp's own strip
// holds the previous DP row.  The recurrence, tie-breaks and output are those of
// the search's alignment phase; queries are read as ASCII from the caller's buffer.
__global__ void __launch_bounds__(128) k_banded_sw_static(
    StaticScratch *__restrict__ scr, const gn_hsp *__restrict__ hsps, uint32_t n, const uint8_t *__restrict__ qascii,
    const uint64_t *__restrict__ qstart, uint32_t n_queries, uint32_t n_seqs, const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
    const uint64_t *__restrict__ seq_start, int32_t match, int32_t mismatch, int32_t go, int32_t ge, int32_t w,
    gn_hit *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    StaticCell *row = scr->strips + (size_t)warp * kStaticSlot;
    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(&scr->next_task, 1u);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= n) return;
        const gn_hsp h = hsps[task];
        if (h.query >= n_queries || h.seq >= n_seqs) {
            if (lane == 0) {
                atomicOr(&scr->status, kErrBadRecord);
                gn_hit z{};
                out[task] = z;
            }
            continue;
        }
        const uint64_t qb = qstart[h.query], sb = seq_start[h.seq];
        const int64_t m = (int64_t)(qstart[h.query + 1] - qb), L = (int64_t)(seq_start[h.seq + 1] - sb);
        const int64_t d_s = (int64_t)h.db_start - h.q_start, d_e = (int64_t)h.db_end - h.q_end;
        const int64_t dlo = min(d_s, d_e) - w, dhi = max(d_s, d_e) + w;
        const int64_t I0 = max((int64_t)0, (int64_t)h.q_start - w), I1 = min(m, (int64_t)h.q_end + w);
        const int64_t J0 = max((int64_t)0, (int64_t)h.db_start - w), J1 = min(L, (int64_t)h.db_end + w);
        const int64_t B = dhi - dlo + 1;
        gn_hit res;
        res.query = h.query; res.seq = h.seq;
        res.q_start = res.q_end = res.db_start = res.db_end = 0;
        res.score = 0; res.rank = 0; res.evalue = 0.0; res.bits = 0.0;
        if (B > kStaticMaxBand || I1 - I0 > 65535) {
            if (lane == 0) { atomicOr(&scr->status, kErrTooWide); out[task] = res; }
            continue;
        }
        int32_t best = 0;
        int64_t bi = INT64_MAX, bj = INT64_MAX;
        uint32_t bs = 0;
        const int32_t goe = go + ge;
        for (int64_t i = I0; i < I1; ++i) {
            const int64_t blo = max((int64_t)0, J0 - i - dlo), bhi = min(B - 1, J1 - 1 - i - dlo);
            if (blo > bhi) continue;
            const bool prow = i - 1 >= I0;
            const int64_t pblo = max((int64_t)0, J0 - (i - 1) - dlo), pbhi = min(B - 1, J1 - 1 - (i - 1) - dlo);
            const uint32_t qc = ascii_code(qascii[qb + (uint64_t)i]);
            int32_t carry_v = kXNeg;
            uint32_t carry_s = 0;
            for (int64_t c0 = blo; c0 <= bhi; c0 += 32) {
                const int64_t b = c0 + lane;
                const bool act = b <= bhi;
                StaticCell pd{0, kNeg, 0, 0}, pu{0, kNeg, 0, 0};
                const bool ok_d = act && prow && b >= pblo && b <= pbhi;
                const bool ok_u = act && prow && b + 1 >= pblo && b + 1 <= pbhi;
                if (ok_d) pd = row[b];
                if (ok_u) pu = row[b + 1];
                __syncwarp();
                int32_t E = kNeg;
                uint32_t SE = 0;
                if (ok_u) {
                    int32_t eo = pu.H + goe, ee = pu.E + ge;
                    if (eo >= ee) { E = eo; SE = pu.SH; } else { E = ee; SE = pu.SE; }
                }
                const int32_t Hd = ok_d ? pd.H : 0;
                const uint32_t SD = (Hd > 0) ? pd.SH : ((uint32_t)(i - I0) << 16) | (uint32_t)b;
                const int64_t j = i + dlo + b;
                int32_t sigma = mismatch;
                if (act) sigma = pair_score(qc, dev_base(bpk, bnb, sb + (uint64_t)j), match, mismatch);
                const int32_t Dg = Hd + sigma;
                int32_t cand;
                uint32_t Sc;
                if (Dg >= E) { cand = Dg; Sc = SD; } else { cand = E; Sc = SE; }
                const int32_t H0 = cand > 0 ? cand : 0;
                int32_t xv = act ? H0 + goe - ge * (int32_t)b : kXNeg;
                uint32_t xs = Sc;
                scan_max_later_wins(xv, xs, lane);
                int32_t ev = __shfl_up_sync(0xffffffffu, xv, 1);
                uint32_t es = __shfl_up_sync(0xffffffffu, xs, 1);
                if (lane == 0) { ev = carry_v; es = carry_s; }
                else if (carry_v > ev) { ev = carry_v; es = carry_s; }
                const int32_t last_v = __shfl_sync(0xffffffffu, xv, 31);
                const uint32_t last_s = __shfl_sync(0xffffffffu, xs, 31);
                if (last_v >= carry_v) { carry_v = last_v; carry_s = last_s; }
                const int32_t F = (ev > kXNeg) ? ev + ge * (int32_t)(b - 1) : kNeg;
                int32_t H;
                uint32_t SH;
                if (H0 >= F) { H = H0; SH = Sc; } else { H = F; SH = es; }
                if (act) {
                    StaticCell c;
                    c.H = H; c.E = E; c.SH = SH; c.SE = SE;
                    row[b] = c;
                    if (H > best) { best = H; bi = i; bj = j; bs = SH; }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            int32_t ob = __shfl_down_sync(0xffffffffu, best, o);
            int64_t oi = __shfl_down_sync(0xffffffffu, bi, o);
            int64_t oj = __shfl_down_sync(0xffffffffu, bj, o);
            uint32_t os = __shfl_down_sync(0xffffffffu, bs, o);
            if (ob > best || (ob == best && (oi < bi || (oi == bi && oj < bj)))) {
                best = ob; bi = oi; bj = oj; bs = os;
            }
        }
        if (lane == 0) {
            if (best > 0) {
                int64_t i0 = I0 + (int64_t)(bs >> 16);
                int64_t j0 = i0 + dlo + (int64_t)(bs & 0xFFFFu);
                res.q_start = (uint32_t)i0; res.q_end = (uint32_t)(bi + 1);
                res.db_start = (uint32_t)j0; res.db_end = (uint32_t)(bj + 1);
                res.score = best;
            }
            out[task] = res;
        }
        __syncwarp();
    }
}

// Device address of g_static_scratch, looked up once per device.
std::mutex g_static_mu;
StaticScratch *g_static_ptr[64] = {nullptr};

StaticScratch *static_scratch(int device) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    GN_REQUIRE(device >= 0 && device < 64, GN_EINVAL, "device ordinal out of range");
    if (!g_static_ptr[device]) {
        void *p = nullptr;
        GN_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_ptr[device] = static_cast<StaticScratch *>(p);
    }
    return g_static_ptr[device];
}

}  // namespace

// Host side of gn_align_hsps_static (see include/genoogle.h).
void align_hsps_static(const gn_index *ix, const char *qbases, const uint64_t *qstart, uint32_t n_queries,
                       const gn_hsp *hsps, uint32_t n, const gn_scoring *sc, uint32_t band_w, gn_hit *out,
                       cudaStream_t s) {
    GN_REQUIRE(ix, GN_EINVAL, "index is required");
    GN_REQUIRE(band_w <= (uint32_t)(kStaticMaxBand - 1) / 2, GN_ETOOBIG,
               "band_w too large for the static scratch (2*band_w+1 must be <= 1024)");
    GN_REQUIRE(n == 0 || (qstart && hsps && out && qbases), GN_EINVAL,
               "query bases and starts, HSPs and output are required");
    GN_REQUIRE(n_queries > 0 || n == 0, GN_EINVAL, "HSPs given without queries");
    gn_scoring d;
    gn_default_params(&d, nullptr);
    const gn_scoring &S = sc ? *sc : d;
    int dev = 0;
    GN_CUDA(cudaGetDevice(&dev));
    GN_REQUIRE(dev == ix->device, GN_EINVAL, "the current device is not the index's device");
    StaticScratch *scr = static_scratch(dev);
    if (n == 0) return;
    // the header must start at zero on every call; strips need no clearing
    GN_CUDA(cudaMemsetAsync(scr, 0, offsetof(StaticScratch, strips), s));
    k_banded_sw_static<<<kStaticWarps * 32 / 128, 128, 0, s>>>(
        scr, hsps, n, reinterpret_cast<const uint8_t *>(qbases), qstart, n_queries, ix->n_seqs, ix->bank.pk, ix->bank.nb, ix->seq_start_d,
        S.match, S.mismatch, S.gap_open, S.gap_extend, (int32_t)band_w, out);
    GN_CUDA(cudaGetLastError());
    uint32_t status = 0;
    GN_CUDA(cudaMemcpyAsync(&status, &scr->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    GN_REQUIRE(!(status & kErrBadRecord), GN_EINVAL,
               "an HSP names a query or bank sequence that does not exist; its record was zeroed");
    GN_REQUIRE(!(status & kErrTooWide), GN_ETOOBIG,
               "an HSP's band spans more than 1024 diagonals (or its window more than 65,535 rows); "
               "its record was written with score 0");
}

}  // namespace gn
