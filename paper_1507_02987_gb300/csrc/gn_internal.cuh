// gn_internal.cuh - internal declarations shared by the CUDA translation units of
// the Genoogle search path (device data layout, primitives, error plumbing).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "genoogle.h"

namespace gn {

// ------------------------------------------------------------------ errors --
struct Error {
    gn_status status;
    std::string msg;
};

void set_error(gn_status st, const std::string &msg);

#define GN_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) {                                                               \
            throw ::gn::Error{_e == cudaErrorMemoryAllocation ? GN_ENOMEM : GN_ECUDA,          \
                              std::string(#call) + ": " + cudaGetErrorString(_e)};             \
        }                                                                                      \
    } while (0)

#define GN_CHECK_LAUNCH() GN_CUDA(cudaGetLastError())

// ------------------------------------------------------ kernel timing --
// When a search runs with GN_FLAG_TIME_KERNELS, every launch made through
// GN_LAUNCH is bracketed by CUDA events on its stream; `units` is the number
// of work items the launch processed (keys, hits, HSPs, cells...).
struct KernelRecord {
    const char *name;
    cudaEvent_t a, b;
    uint64_t units;
};
struct KernelTimer {
    std::vector<KernelRecord> recs;
    ~KernelTimer() {
        for (auto &r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
};
extern thread_local KernelTimer *g_ktimer;
void count_launch();

#define GN_LAUNCH(name, units, stream, ...)                                        \
    do {                                                                           \
        ::gn::KernelTimer *_kt = ::gn::g_ktimer;                                   \
        cudaEvent_t _ea = nullptr, _eb = nullptr;                                  \
        if (_kt && cudaEventCreate(&_ea) == cudaSuccess) cudaEventRecord(_ea, stream); \
        __VA_ARGS__;                                                               \
        GN_CHECK_LAUNCH();                                                         \
        ::gn::count_launch();                                                      \
        if (_ea && cudaEventCreate(&_eb) == cudaSuccess) {                         \
            cudaEventRecord(_eb, stream);                                          \
            _kt->recs.push_back({(name), _ea, _eb, (uint64_t)(units)});            \
        } else if (_ea) {                                                          \
            cudaEventDestroy(_ea);                                                 \
        }                                                                          \
    } while (0)

#define GN_REQUIRE(cond, st, msg)                 \
    do {                                          \
        if (!(cond)) throw ::gn::Error{(st), (msg)}; \
    } while (0)

// Device-side status word bits (kernels record a failed check and skip the access).
enum : uint32_t {
    DEV_ERR_BAND_TOO_WIDE = 1u,   // alignment band wider than the start encoding allows
    DEV_ERR_CAPACITY = 2u,        // an output buffer was too small (caller retries with more room)
    DEV_ERR_BOUNDS = 4u,          // an index fell outside its buffer
    DEV_ERR_TIMEOUT = 8u,         // a bounded device-side wait ran out
};

// ------------------------------------------------------------- constants --
constexpr uint32_t QBIAS = 65536;          // > any query offset: diagonal key = gpos - qpos + QBIAS > 0
constexpr uint32_t MAX_QUERY_LEN = 65535;   // longest query (segment) the seed phases take
constexpr uint64_t MAX_LONG_QUERY_LEN = (1ull << 24) - 1;  // longest query gn_search takes (in segments)
constexpr uint32_t SEG_OVERLAP = 8192;      // bases shared by neighbouring segments of a long query
constexpr uint32_t SEG_STEP = MAX_QUERY_LEN - SEG_OVERLAP;
constexpr uint32_t MAX_QUERIES = 65536;
constexpr uint64_t HIT_BYTES = 24;  // device bytes budgeted per raw hit of a query chunk

// --------------------------------------------------------- device memory --
// Stream-ordered allocations from the device's default memory pool.
class DeviceArena {
public:
    explicit DeviceArena(cudaStream_t s) : stream_(s) {}
    ~DeviceArena() { release(); }
    void *alloc(size_t bytes);
    template <class T> T *alloc_n(size_t n) { return static_cast<T *>(alloc(sizeof(T) * (n ? n : 1))); }
    void release();
    cudaStream_t stream() const { return stream_; }

private:
    cudaStream_t stream_;
    std::vector<void *> ptrs_;
};

void configure_mempool(int device);

// Integer-pipe throughput (gn_measure_int_peaks).
void measure_int_peaks(gn_int_peaks *out, cudaStream_t s);

// Allocation fault injection and counters (tests): see gn_debug_fail_alloc.
void debug_fail_alloc(uint64_t nth);
uint64_t debug_alloc_count();
int64_t debug_live_allocs();

// ------------------------------------------------------------ packed DNA --
// 16 bases per uint32 word, first base in the two most significant bits;
// a parallel bitmap marks non-bases (bit g & 31 of word g >> 5).  One extra
// zero word is kept at the end of both arrays so windows can read word w + 1.
struct Packed {
    uint32_t *pk = nullptr;
    uint32_t *nb = nullptr;
    uint64_t n = 0;
    static uint64_t pk_words(uint64_t n) { return (n + 15) / 16 + 2; }
    static uint64_t nb_words(uint64_t n) { return (n + 31) / 32 + 2; }
};

void pack_bases(const uint8_t *ascii_dev, uint64_t n, Packed &out, cudaStream_t s);

// --------------------------------------------------------------- scans --
// out[i] = sum(in[0..i)), out[n] = total; out has n + 1 entries.  One pass over the data
// (decoupled look-back); a wait that runs out records DEV_ERR_TIMEOUT in *g_wait_status
// (the calling thread's current search or index build) when it is set.
size_t scan_scratch_bytes(uint64_t n);
void exclusive_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, void *scratch, cudaStream_t s);
extern thread_local uint32_t *g_wait_status;
bool debug_scan(const uint32_t *in, uint64_t *out, uint64_t n, long long budget, int drop_first, cudaStream_t s);
// Sets g_wait_status for the scope (a device word the caller checks for DEV_ERR_TIMEOUT).
struct WaitStatusScope {
    uint32_t *prev;
    explicit WaitStatusScope(uint32_t *w) : prev(g_wait_status) { g_wait_status = w; }
    ~WaitStatusScope() { g_wait_status = prev; }
};

// ----------------------------------------------------------- radix sort --
// Stable LSD radix sort of 64-bit keys (optionally carrying 32-bit values) on
// key bits [bit_lo, bit_hi).  Ping-pongs between the two buffers; returns true
// when the sorted data ended in the *_alt buffers.
size_t radix_scratch_bytes(uint64_t n);
struct RadixTag {
    const char *up, *down;     // kernel-timer names: histogram and pass kernels of the single-pass sort
    const char *up3, *down3;   // upsweep and downsweep of the three-kernel passes (large sorts)
};
extern const RadixTag TAG_HIT_SORT, TAG_INDEX_SORT, TAG_RECORD_SORT;
bool radix_sort(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint64_t n, int bit_lo,
                int bit_hi, void *scratch, cudaStream_t s, const RadixTag &tag);
bool debug_sort(uint64_t *keys, uint32_t *vals, uint64_t n, int bit_lo, int bit_hi, long long budget,
                int drop_first, bool three_kernel, cudaStream_t s);
unsigned long long launch_count();

// Sort of fixed-size records made of uint32 words by a list of fields (first =
// most significant).  Produces the permutation perm (record ids in order).
struct SortField {
    int word;   // word index inside the record
    int bits;   // significant bits of the field
    bool desc;  // descending order
};
void sort_records(const uint32_t *recs, int rec_words, uint32_t n, const std::vector<SortField> &fields,
                  uint32_t *perm_out, DeviceArena &arena, cudaStream_t s);

// Gathers records by a permutation: out[i] = in[perm[i]].
void gather_records(const uint32_t *in, int rec_words, const uint32_t *perm, uint32_t n, uint32_t *out,
                    cudaStream_t s);

int bits_for(uint64_t max_value);  // bits needed to hold values in [0, max_value]

int num_sms();

// Compacts records whose flag is non-zero, keeping their order; returns the count
// (synchronizes the stream to read it).
uint32_t compact_records(const uint32_t *in, int rec_words, const uint32_t *flags, uint32_t n, uint32_t *out,
                         DeviceArena &arena, cudaStream_t s);

// ------------------------------------------------------- device helpers --
__device__ __forceinline__ uint32_t dev_kmer(const uint32_t *__restrict__ pk, uint64_t g, int k) {
    uint64_t w = g >> 4;
    int off = (int)(g & 15);
    uint64_t v = ((uint64_t)pk[w] << 32) | (uint64_t)pk[w + 1];
    v <<= 2 * off;
    return (uint32_t)(v >> (64 - 2 * k));
}

__device__ __forceinline__ bool dev_has_nonbase(const uint32_t *__restrict__ nb, uint64_t g, int k) {
    uint64_t w = g >> 5;
    int off = (int)(g & 31);
    uint64_t v = ((uint64_t)nb[w + 1] << 32) | (uint64_t)nb[w];
    v >>= off;
    return (v & ((1ull << k) - 1ull)) != 0ull;
}

// Seed shape: a seed covers `span` (<= 32) consecutive bases and keeps those whose bit
// is set in `keep` (k of them, k <= 16); its code is the kept bases in order, first
// most significant.  A plain k-mer is span = k with every bit kept.
struct SeedShape {
    int k, span;
    uint32_t keep;
};

__device__ __forceinline__ uint32_t dev_seed_code(const uint32_t *__restrict__ pk, uint64_t g, const SeedShape &sh) {
    if (sh.span == sh.k) return dev_kmer(pk, g, sh.k);
    const uint64_t w = g >> 4;
    const int off = (int)(g & 15);
    const uint64_t hi = ((uint64_t)pk[w] << 32) | (uint64_t)pk[w + 1];
    const uint64_t v = off ? (hi << (2 * off)) | ((uint64_t)pk[w + 2] >> (32 - 2 * off)) : hi;  // bases g .. g+31
    uint32_t code = 0, m = sh.keep;
    while (m) {
        const int p = __ffs(m) - 1;
        m &= m - 1;
        code = (code << 2) | (uint32_t)((v >> (62 - 2 * p)) & 3u);
    }
    return code;
}

__device__ __forceinline__ bool dev_seed_has_nonbase(const uint32_t *__restrict__ nb, uint64_t g, const SeedShape &sh) {
    const uint64_t w = g >> 5;
    const int off = (int)(g & 31);
    const uint64_t v = (((uint64_t)nb[w + 1] << 32) | (uint64_t)nb[w]) >> off;
    return (v & (uint64_t)sh.keep) != 0ull;
}

// 2-bit code of base g, or 4 for a non-base
__device__ __forceinline__ uint32_t dev_base(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb,
                                             uint64_t g) {
    uint32_t bad = (nb[g >> 5] >> (g & 31)) & 1u;
    uint32_t c = (pk[g >> 4] >> (30 - 2 * (int)(g & 15))) & 3u;
    return bad ? 4u : c;
}

// last index s in [0, n) with a[s] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ uint32_t dev_upper_index(const uint64_t *__restrict__ a, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;  // invariant: a[lo] <= x, a[hi] > x (hi == n: past the end)
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Sequence lookup: lut[j] is the sequence holding bank position j << SEQ_LUT_SHIFT, so
// the sequence of position x is found by a short forward walk from lut[x >> shift]
// (sequences of >= 1 base; a block of 2^SEQ_LUT_SHIFT bases starts few of them).
// Entries allocated for n occurrences: whole quads (16 bytes), so that the search may read
// any list in aligned 16-byte loads; the entries past n are never used.
inline uint64_t post_alloc_entries(uint64_t n) { return std::max<uint64_t>(4, (n + 3) & ~3ull); }

constexpr int SEQ_LUT_SHIFT = 10;
struct SeqMap {
    const uint64_t *start;  // n_seqs + 1 sequence starts (start[n_seqs] = bank length)
    const uint32_t *lut;
    uint32_t n_seqs;
};
// ------------------------------------------------------ device-side checks --
// Built with -DGN_CHECKS (paper_1507_02987_gb300._build.build(checks=True)), the search
// kernels check indices they compute from data before using them; a failed check records
// DEV_ERR_BOUNDS in g_check_bits and skips the access, and the search then returns
// GN_EINTERNAL.  Without it the checks compile to nothing.
#ifdef GN_CHECKS
static __device__ uint32_t g_check_bits;
#define GN_CHECK(cond) ((cond) || (atomicOr(&::gn::g_check_bits, (uint32_t)DEV_ERR_BOUNDS), false))
#else
#define GN_CHECK(cond) true
#endif

// sequence holding bank position x (x < bank length); empty sequences are skipped
__device__ __forceinline__ uint32_t dev_seq_of(const SeqMap &m, uint64_t x) {
    if (!GN_CHECK(x < m.start[m.n_seqs])) return m.n_seqs ? m.n_seqs - 1 : 0u;
    uint32_t s = m.lut[x >> SEQ_LUT_SHIFT];
    while (m.start[s + 1] <= x) ++s;
    return s;
}

}  // namespace gn

// --------------------------------------------------------------- handles --
struct gn_index {
    int k = 0, t = 0;
    int span = 0;        // bases a seed covers (k without a mask)
    gn_tuning tuning{};  // result-invariant execution settings (0 = defaults)
    uint32_t keep = 0;   // kept positions of a seed (all k bits without a mask)
    int device = 0;
    uint32_t n_seqs = 0;
    uint64_t n_bases = 0;
    uint64_t n_postings = 0;
    uint32_t max_seq_len = 0;
    std::vector<uint64_t> seq_start_h;
    uint64_t *seq_start_d = nullptr;  // n_seqs + 1
    uint32_t *seq_lut_d = nullptr;    // (n_bases >> SEQ_LUT_SHIFT) + 1 entries, see SeqMap
    gn::Packed bank;                  // packed bank + non-base bitmap
    uint64_t *off_d = nullptr;        // 4^k + 1 bucket starts
    uint32_t *post_d = nullptr;       // occurrences: global base offset of the window (post_alloc_entries)
    uint64_t device_bytes = 0;
    // per-phase device times of the most recent search through this handle
    std::vector<std::pair<const char *, float>> last_phases;
    struct KernelStat {
        const char *name;
        double ms;
        uint32_t launches;
        uint64_t units;
    };
    std::vector<KernelStat> last_kernels;
    std::mutex phase_mu;
};

struct gn_results {
    uint32_t n_queries = 0;
    std::vector<uint64_t> qoff;  // n_queries + 1
    std::vector<gn_hit> hits;
    bool has_stages = false;
    std::vector<gn_hsp> st_hsp, st_ext, st_merged, st_sel;
    std::vector<gn_hit> st_aln;
    std::vector<uint32_t> st_hits;     // quadruples (query, qpos, seq, pos)
    std::vector<uint64_t> st_hit_counts;
};

namespace gn {
void index_build(const gn_bank *db, int k, int stride, cudaStream_t s, gn_index *ix);
void index_build_masked(const gn_bank *db, const char *mask, int stride, cudaStream_t s, gn_index *ix);
void index_free(gn_index *ix);
void index_export(const gn_index *ix, uint64_t *bucket_start, uint32_t *post_seq, uint32_t *post_pos);
void index_save(const gn_index *ix, const char *path);
void index_load(const char *path, gn_index *ix);

inline SeqMap seq_map(const gn_index *ix) { return SeqMap{ix->seq_start_d, ix->seq_lut_d, ix->n_seqs}; }
inline SeedShape seed_shape(const gn_index *ix) { return SeedShape{ix->k, ix->span, ix->keep}; }

// Seed hits of each of n queries (ASCII bases and starts in device memory): hits[q] is the
// sum of the occurrence-list lengths of query q's seed codes (request admission).
void count_request_hits(const gn_index *ix, const uint8_t *bases, const uint64_t *start, uint32_t n,
                        unsigned long long *hits, cudaStream_t s);
struct SearchOptions {
    gn_scoring sc;
    gn_params p;           // resolved (no zero defaults left)
    uint64_t mem_cap = 0;  // device bytes the hit storage of one query chunk may take (0: 55 % of free)
    uint64_t max_hit_bytes = 0;  // GN_ETOOBIG if the call's hits need more (HIT_BYTES each; 0: no limit)
};
// Query i -> queries 2i (as given) and 2i + 1 (reverse complement) in device memory from arena.
void both_strands(const uint8_t *qbases_dev, const std::vector<uint64_t> &qstart_h, DeviceArena &arena,
                  cudaStream_t s, const uint8_t **out_bases, std::vector<uint64_t> &out_start);
// Device-resident query set: bases (ASCII) on the device, starts on the host.
void search(gn_index *ix, const uint8_t *qbases_dev, const std::vector<uint64_t> &qstart, const SearchOptions &o,
            cudaStream_t s, gn_results *res);
void align_hsps_static(const gn_index *ix, const char *qbases, const uint64_t *qstart, uint32_t n_queries,
                       const gn_hsp *hsps, uint32_t n, const gn_scoring *sc, uint32_t band_w, gn_hit *out,
                       cudaStream_t s);
}  // namespace gn
