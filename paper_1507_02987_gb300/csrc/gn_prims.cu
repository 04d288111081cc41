// gn_prims.cu - device primitives of the search path: 2-bit packing, exclusive
// scans, a stable LSD radix sort and record sorting built on it.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "gn_internal.cuh"

namespace gn {

// ------------------------------------------------------------- helpers --
int bits_for(uint64_t max_value) {
    int b = 0;
    while (b < 64 && (max_value >> b) != 0) ++b;
    return b;
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

void configure_mempool(int device) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    GN_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;  // keep freed blocks in the pool: repeated searches reuse them
    GN_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    done[device] = true;
}

// Allocation fault injection (tests): the n-th next arena allocation fails as if the device
// were out of memory.  Counters of arena allocations made and held.
static std::atomic<uint64_t> g_fail_alloc_in{0};
static std::atomic<uint64_t> g_alloc_count{0};
static std::atomic<int64_t> g_live_allocs{0};

void debug_fail_alloc(uint64_t nth) { g_fail_alloc_in.store(nth); }
uint64_t debug_alloc_count() { return g_alloc_count.load(); }
int64_t debug_live_allocs() { return g_live_allocs.load(); }

void *DeviceArena::alloc(size_t bytes) {
    uint64_t v = g_fail_alloc_in.load();
    while (v && !g_fail_alloc_in.compare_exchange_weak(v, v - 1)) {
    }
    if (v == 1) throw Error{GN_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)"};
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 1, stream_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{GN_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                   cudaGetErrorString(e)};
    }
    ptrs_.push_back(p);
    g_alloc_count.fetch_add(1);
    g_live_allocs.fetch_add(1);
    return p;
}

void DeviceArena::release() {
    for (void *p : ptrs_) cudaFreeAsync(p, stream_);
    g_live_allocs.fetch_sub((int64_t)ptrs_.size());
    ptrs_.clear();
}

// --------------------------------------------------------------- packing --
__device__ __forceinline__ uint32_t base_bits(uint32_t b, uint32_t &bad) {
    uint32_t c = b & 0xDFu;  // upper case for letters; other bytes stay non-bases
    uint32_t code = (c == 'C') ? 1u : (c == 'G') ? 2u : (c == 'T' || c == 'U') ? 3u : 0u;
    bad = (c == 'A' || c == 'C' || c == 'G' || c == 'T' || c == 'U') ? 0u : 1u;
    return code;
}

// One thread packs 32 bases: two code words and one non-base word.
__global__ void k_pack(const uint8_t *__restrict__ ascii, uint64_t n, uint32_t *__restrict__ pk,
                       uint32_t *__restrict__ nb, int aligned16) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t g0 = t * 32;
    if (g0 >= n) return;
    uint8_t buf[32];
    if (aligned16 && g0 + 32 <= n) {
        const uint4 *src = reinterpret_cast<const uint4 *>(ascii + g0);
        uint4 a = __ldg(src), b = __ldg(src + 1);
        memcpy(buf, &a, 16);
        memcpy(buf + 16, &b, 16);
    } else {
        for (int i = 0; i < 32; ++i) buf[i] = (g0 + i < n) ? ascii[g0 + i] : (uint8_t)'N';
    }
    uint32_t w0 = 0, w1 = 0, bw = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        uint32_t bad;
        uint32_t c = base_bits(buf[i], bad);
        if (i < 16) w0 |= c << (30 - 2 * i);
        else w1 |= c << (30 - 2 * (i - 16));
        bw |= bad << i;
    }
    pk[2 * t] = w0;
    pk[2 * t + 1] = w1;
    nb[t] = bw;
}

void pack_bases(const uint8_t *ascii_dev, uint64_t n, Packed &out, cudaStream_t s) {
    out.n = n;
    GN_CUDA(cudaMemsetAsync(out.pk, 0, Packed::pk_words(n) * 4, s));
    GN_CUDA(cudaMemsetAsync(out.nb, 0xFF, Packed::nb_words(n) * 4, s));
    if (n == 0) return;
    uint64_t threads = (n + 31) / 32;
    int aligned = ((uintptr_t)ascii_dev % 16) == 0;
    GN_LAUNCH("k_pack", n, s,
              k_pack<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(ascii_dev, n, out.pk, out.nb, aligned));
}

// ----------------------------------------------------------------- scans --

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; returns the block total in *total.
template <class T, int THREADS>
__device__ __forceinline__ T block_excl_scan(T v, T *warp_sums, T *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        T x = (lane < THREADS / 32) ? warp_sums[lane] : T(0);
        T xi = warp_incl_scan(x);
        if (lane < THREADS / 32) warp_sums[lane] = xi - x;
        if (lane == THREADS / 32 - 1) *total = xi;
    }
    __syncthreads();
    T r = inc - v + warp_sums[w];
    __syncthreads();
    return r;
}

// Single-pass scan with decoupled look-back.  A block takes the next tile from a ticket
// counter (so every tile it waits on belongs to a block that is already running), sums
// it, publishes the sum in the tile's state word, then its first warp reads the states of
// the preceding tiles 32 at a time, adding sums until it meets a tile whose inclusive
// prefix is published; the block then publishes its own inclusive prefix and writes its
// outputs.  A state word holds a flag in its top two bits (0: nothing yet, 1: the tile's
// sum, 2: its inclusive prefix) and the value below.  The wait for a predecessor's state
// is bounded: after `budget` SM clock cycles the block records DEV_ERR_TIMEOUT in
// *status, takes the prefix found so far and goes on (its outputs are then wrong, and
// the caller reports the error).
constexpr int SP_THREADS = 256, SP_ITEMS = 8, SP_TILE = SP_THREADS * SP_ITEMS;
constexpr uint64_t SP_AGG = 1ull << 62, SP_PRE = 2ull << 62, SP_VAL = (1ull << 62) - 1;

__global__ void __launch_bounds__(SP_THREADS) k_scan_onepass(const uint32_t *__restrict__ in, uint64_t n,
                                                             uint64_t *__restrict__ out, uint32_t *ticket,
                                                             unsigned long long *state, uint32_t *status,
                                                             long long budget, int drop_first) {
    __shared__ uint32_t tin[SP_TILE + SP_TILE / 32];  // one pad word per 32: conflict-free runs
    __shared__ uint64_t tout[SP_TILE + SP_TILE / 32];
    __shared__ uint64_t ws[SP_THREADS / 32];
    __shared__ uint64_t s_tot, s_prefix;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    const uint64_t base = (uint64_t)t * SP_TILE;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
        const int li = j * SP_THREADS + tid;
        tin[li + (li >> 5)] = base + li < n ? in[base + li] : 0u;
    }
    __syncthreads();
    uint64_t loc[SP_ITEMS];
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
        const int li = tid * SP_ITEMS + j;
        loc[j] = sum;
        sum += tin[li + (li >> 5)];
    }
    const uint64_t off = block_excl_scan<uint64_t, SP_THREADS>(sum, ws, &s_tot);
    if (tid < 32) {
        const uint64_t agg = s_tot;
        uint64_t excl = 0;
        if (t == 0) {
            if (lane == 0 && !drop_first) atomicExch(&state[0], SP_PRE | agg);
        } else {
            if (lane == 0) atomicExch(&state[t], SP_AGG | agg);
            int64_t j = (int64_t)t - 1;
            const long long t0 = clock64();
            for (;;) {
                const int64_t q = j - lane;
                const uint64_t st = q >= 0 ? *(volatile unsigned long long *)&state[q] : SP_PRE;
                // lanes up to the nearest published prefix must all hold a state
                const uint32_t pre = __ballot_sync(0xffffffffu, (st >> 62) == 2ull);
                const uint32_t none = __ballot_sync(0xffffffffu, (st >> 62) == 0ull);
                const int stop = pre ? __ffs(pre) - 1 : 31;
                const uint32_t need = stop == 31 ? 0xffffffffu : (2u << stop) - 1u;
                if (none & need) {
                    if (clock64() - t0 > budget) {
                        if (lane == 0) atomicOr(status, DEV_ERR_TIMEOUT);
                        break;
                    }
                    continue;
                }
                uint64_t v = lane <= stop ? (st & SP_VAL) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                excl += __shfl_sync(0xffffffffu, v, 0);
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) atomicExch(&state[t], SP_PRE | (excl + agg));
        }
        if (lane == 0) s_prefix = excl;
    }
    __syncthreads();
    const uint64_t pre = s_prefix + off;
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
        const int li = tid * SP_ITEMS + j;
        tout[li + (li >> 5)] = pre + loc[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SP_ITEMS; ++j) {
        const int li = j * SP_THREADS + tid;
        if (base + li < n) out[base + li] = tout[li + (li >> 5)];
    }
    if (base + SP_TILE >= n && tid == 0) out[n] = s_prefix + s_tot;  // the last tile: the total
}

// One block scans up to SC_SMALL elements: each thread sums a contiguous run, the block
// scans the run totals, then each thread writes its run's prefixes.
constexpr uint64_t SC_SMALL = 4096;

__global__ void __launch_bounds__(1024) k_scan_small(const uint32_t *__restrict__ in, uint64_t n,
                                                     uint64_t *__restrict__ out) {
    constexpr int T = 1024;
    __shared__ uint64_t ws[T / 32];
    __shared__ uint64_t tot;
    const uint64_t per = (n + T - 1) / T;
    const uint64_t b = threadIdx.x * per, e = min(n, b + per);
    uint64_t s = 0;
    for (uint64_t i = b; i < e; ++i) s += in[i];
    uint64_t off = block_excl_scan<uint64_t, T>(s, ws, &tot);
    for (uint64_t i = b; i < e; ++i) {
        const uint64_t v = in[i];
        out[i] = off;
        off += v;
    }
    if (threadIdx.x == 0) out[n] = tot;
}

// Scratch of one scan: ticket counter, status word, tile states.
size_t scan_scratch_bytes(uint64_t n) { return 16 + sizeof(uint64_t) * ((n + SP_TILE - 1) / SP_TILE + 1); }

// Bound of the scan's wait for a preceding tile, in SM clock cycles: about a second.
constexpr long long SCAN_WAIT_BUDGET = 1ll << 31;
thread_local uint32_t *g_wait_status = nullptr;

static void scan_onepass(const uint32_t *in, uint64_t *out, uint64_t n, void *scratch, uint32_t *status,
                         long long budget, int drop_first, cudaStream_t s) {
    const uint64_t nb = (n + SP_TILE - 1) / SP_TILE;
    uint32_t *head = static_cast<uint32_t *>(scratch);
    unsigned long long *state = reinterpret_cast<unsigned long long *>(head + 4);
    GN_CUDA(cudaMemsetAsync(scratch, 0, 16 + 8 * nb, s));
    GN_LAUNCH("k_scan_onepass", n, s,
              k_scan_onepass<<<(unsigned)nb, SP_THREADS, 0, s>>>(in, n, out, head, state,
                                                               status ? status : head + 1, budget, drop_first));
}

void exclusive_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, void *scratch, cudaStream_t s) {
    if (n == 0) {
        GN_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
        return;
    }
    if (n <= SC_SMALL) {
        GN_LAUNCH("k_scan_small", n, s, k_scan_small<<<1, 1024, 0, s>>>(in, n, out));
        return;
    }
    scan_onepass(in, out, n, scratch, g_wait_status, SCAN_WAIT_BUDGET, 0, s);
}

// Scan of caller buffers with a given wait budget; drop_first keeps the first tile from
// publishing its state, so that the next tiles' waits run out.  Returns whether a wait ran out.
bool debug_scan(const uint32_t *in, uint64_t *out, uint64_t n, long long budget, int drop_first, cudaStream_t s) {
    DeviceArena arena(s);
    void *scr = arena.alloc(scan_scratch_bytes(n));
    uint32_t *st = arena.alloc_n<uint32_t>(1);
    GN_CUDA(cudaMemsetAsync(st, 0, 4, s));
    if (n == 0) GN_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    else scan_onepass(in, out, n, scr, st, budget, drop_first, s);
    uint32_t h = 0;
    GN_CUDA(cudaMemcpyAsync(&h, st, 4, cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    return (h & DEV_ERR_TIMEOUT) != 0;
}

// ------------------------------------------------------------ radix sort --
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_MAX_GRID_PER_SM = 8;

__global__ void __launch_bounds__(RS_THREADS) k_rs_upsweep(const uint64_t *__restrict__ keys, uint64_t n,
                                                           uint64_t chunk, int shift, uint32_t mask,
                                                           uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    uint64_t beg = (uint64_t)blockIdx.x * chunk, end = min(n, beg + chunk);
    uint64_t i = beg + threadIdx.x;
    for (; i + 3 * RS_THREADS < end; i += 4 * RS_THREADS) {
        uint64_t k0 = keys[i], k1 = keys[i + RS_THREADS], k2 = keys[i + 2 * RS_THREADS], k3 = keys[i + 3 * RS_THREADS];
        atomicAdd(&h[w][(uint32_t)(k0 >> shift) & mask], 1u);
        atomicAdd(&h[w][(uint32_t)(k1 >> shift) & mask], 1u);
        atomicAdd(&h[w][(uint32_t)(k2 >> shift) & mask], 1u);
        atomicAdd(&h[w][(uint32_t)(k3 >> shift) & mask], 1u);
    }
    for (; i < end; i += RS_THREADS) atomicAdd(&h[w][(uint32_t)(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) s += h[ww][d];
        counts[(uint64_t)d * gridDim.x + blockIdx.x] = s;
    }
}

struct RsSmem {
    uint32_t wcnt[RS_WARPS][256];
    uint32_t tcnt[256];
    uint32_t tbase[256];
    unsigned long long run[256];
    uint32_t ws[RS_WARPS];
    uint32_t tot;
};

// Ranks one tile of keys (tn <= RS_TILE, starting at tb) by digit and writes them (and
// their values) to sk / sv in digit order, stably: S.tcnt[d] keys of digit d start at
// S.tbase[d].  Keys are read warp-striped (warp w holds tile positions w * 512 to
// w * 512 + 511), ranked per warp with __match_any_sync, and the per-warp counts are
// scanned over the warps, then over the digits.  Ends with the block synchronised.
template <bool VALS>
__device__ __forceinline__ void rs_rank_tile(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                             uint64_t tb, uint32_t tn, int shift, uint32_t mask, RsSmem &S,
                                             uint64_t *sk, uint32_t *sv) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&S.wcnt[0][0])[i] = 0;
    __syncthreads();
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t dg[RS_ITEMS];
    uint32_t rk[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t li = warp * (RS_ITEMS * 32) + it * 32 + lane;
        bool ok = li < tn;
        k[it] = ok ? kin[tb + li] : 0ull;
        if (VALS) v[it] = ok ? vin[tb + li] : 0u;
        dg[it] = ok ? ((uint32_t)(k[it] >> shift) & mask) : 256u;
    }
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t d = dg[it];
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = (d < 256u) ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        rk[it] = before + __popc(peers & lt_mask);
        if (d < 256u && (peers & lt_mask) == 0u) S.wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = tid;  // RS_THREADS == 256 digits
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = S.wcnt[w][d];
            S.wcnt[w][d] = s;
            s += c;
        }
        S.tcnt[d] = s;
        uint32_t b = block_excl_scan<uint32_t, RS_THREADS>(s, S.ws, &S.tot);
        S.tbase[d] = b;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t d = dg[it];
        if (d < 256u) {
            uint32_t pos = S.tbase[d] + S.wcnt[warp][d] + rk[it];
            sk[pos] = k[it];
            if (VALS) sv[pos] = v[it];
        }
    }
    __syncthreads();
}

template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS) k_rs_downsweep(const uint64_t *__restrict__ kin,
                                                             const uint32_t *__restrict__ vin,
                                                             uint64_t *__restrict__ kout,
                                                             uint32_t *__restrict__ vout, uint64_t n,
                                                             uint64_t chunk, int shift, uint32_t mask,
                                                             const uint64_t *__restrict__ offs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RsSmem &S = *reinterpret_cast<RsSmem *>(smem_raw);
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw + ((sizeof(RsSmem) + 15) / 16) * 16);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + RS_TILE);
    const int tid = threadIdx.x;
    if (tid < 256) S.run[tid] = offs[(uint64_t)tid * gridDim.x + blockIdx.x];
    uint64_t beg = (uint64_t)blockIdx.x * chunk, end = min(n, beg + chunk);
    for (uint64_t tb = beg; tb < end; tb += RS_TILE) {
        const uint32_t tn = (uint32_t)min((uint64_t)RS_TILE, end - tb);
        rs_rank_tile<VALS>(kin, vin, tb, tn, shift, mask, S, sk, sv);
        for (uint32_t i = tid; i < tn; i += RS_THREADS) {
            uint64_t key = sk[i];
            uint32_t d = (uint32_t)(key >> shift) & mask;
            uint64_t dst = S.run[d] + (i - S.tbase[d]);
            kout[dst] = key;
            if (VALS) vout[dst] = sv[i];
        }
        __syncthreads();
        S.run[tid] += S.tcnt[tid];
        __syncthreads();
    }
}

// ------------------------------------------------- single-pass radix sort --
// For sorts of up to OS_MAX_TILES tiles: a histogram kernel counts the first pass's digits,
// then one kernel per 8-bit pass.  A block of a pass takes the next tile from the pass's
// ticket counter (so every tile it waits on belongs to a block that is already running),
// turns the pass's digit counts into the digits' starts, ranks the tile's keys by digit,
// counts the next pass's digits of its keys, publishes the tile's count of each digit, and
// each thread (one per digit) adds the counts of the preceding tiles, reading OS_LOOK
// state words at a time, until it meets a tile whose inclusive prefix is published
// (decoupled look-back, as in the scan above); the block then publishes its inclusive
// prefixes and writes its keys to their places.  A state word: flag in bits 63-62 (0
// nothing, 1 the tile's count, 2 its inclusive prefix), the pass (plus one) in bits 61-56,
// the value below; the words of all passes share one array, a word of an earlier pass
// counting as not yet published.  Waits are bounded as in the scan (DEV_ERR_TIMEOUT).
constexpr int OS_MAX_PASSES = 8;
constexpr int OS_LOOK = 16;
constexpr uint64_t OS_MAX_TILES = 1u << 15;
constexpr uint64_t OS_AGG = 1ull << 62, OS_PRE = 2ull << 62, OS_EPOCH = 0x3Full << 56, OS_VAL = (1ull << 56) - 1;

// Digit counts of the first pass (per-warp shared-memory counts, then one global atomic per
// digit and block); each pass counts the next pass's digits of its own keys.
__global__ void __launch_bounds__(RS_THREADS) k_os_hist(const uint64_t *__restrict__ keys, uint64_t n, int shift,
                                                        uint32_t mask, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[RS_WARPS][256];
    const int tid = threadIdx.x, w = tid >> 5;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * RS_THREADS + tid; i < n; i += (uint64_t)gridDim.x * RS_THREADS)
        atomicAdd(&h[w][(uint32_t)(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) c += h[ww][tid];
    if (c) atomicAdd(&hist[tid], c);
}

template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 3) k_os_pass(const uint64_t *__restrict__ kin,
                                                        const uint32_t *__restrict__ vin,
                                                        uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                        uint64_t n, int shift, uint32_t mask, uint64_t epoch,
                                                        const uint32_t *__restrict__ hist,
                                                        uint32_t *__restrict__ next_hist, int next_shift,
                                                        uint32_t next_mask, unsigned long long *state,
                                                        uint32_t *ticket, uint32_t *status, long long budget,
                                                        int drop_first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RsSmem &S = *reinterpret_cast<RsSmem *>(smem_raw);
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw + ((sizeof(RsSmem) + 15) / 16) * 16);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + RS_TILE);
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t tb = (uint64_t)tile * RS_TILE;
    const uint32_t tn = (uint32_t)min((uint64_t)RS_TILE, n - tb);
    // the digits' starts: exclusive scan of the pass's digit counts (complete: the previous
    // launch, or the histogram kernel, counted them)
    const uint32_t dstart = block_excl_scan<uint32_t, RS_THREADS>(hist[tid], S.ws, &S.tot);
    rs_rank_tile<VALS>(kin, vin, tb, tn, shift, mask, S, sk, sv);
    if (next_hist) {  // the next pass's digit counts of this tile's keys
        for (int i = tid; i < 256; i += RS_THREADS) S.wcnt[0][i] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < tn; i += RS_THREADS) atomicAdd(&S.wcnt[0][(uint32_t)(sk[i] >> next_shift) & next_mask], 1u);
        __syncthreads();
        const uint32_t c = S.wcnt[0][tid];
        if (c) atomicAdd(&next_hist[tid], c);
    }
    {
        const uint32_t d = tid;
        const uint64_t cnt = S.tcnt[d];
        unsigned long long *mine = state + (uint64_t)tile * 256 + d;
        uint64_t excl = 0;
        if (tile == 0) {
            if (!drop_first) atomicExch(mine, OS_PRE | epoch | cnt);
        } else {
            atomicExch(mine, OS_AGG | epoch | cnt);
            int64_t j = (int64_t)tile - 1;
            const long long t0 = clock64();
            for (;;) {
                uint64_t w[OS_LOOK];
#pragma unroll
                for (int k = 0; k < OS_LOOK; ++k) {
                    const int64_t q = j - k;
                    w[k] = q >= 0 ? *(volatile unsigned long long *)&state[(uint64_t)q * 256 + d] : (OS_PRE | epoch);
                }
                int used = OS_LOOK;
                bool pre = false;
#pragma unroll
                for (int k = 0; k < OS_LOOK; ++k) {
                    if (used == OS_LOOK && !pre) {
                        const uint64_t x = w[k];
                        if ((x >> 62) == 0ull || (x & OS_EPOCH) != epoch) {
                            used = k;
                        } else {
                            excl += x & OS_VAL;
                            pre = (x >> 62) == 2ull;
                        }
                    }
                }
                if (pre) break;
                j -= used;
                if (used < OS_LOOK && clock64() - t0 > budget) {
                    atomicOr(status, DEV_ERR_TIMEOUT);
                    break;
                }
            }
            atomicExch(mine, OS_PRE | epoch | (excl + cnt));
        }
        S.run[d] = dstart + excl;
    }
    __syncthreads();
    for (uint32_t i = tid; i < tn; i += RS_THREADS) {
        const uint64_t key = sk[i];
        const uint32_t d = (uint32_t)(key >> shift) & mask;
        const uint64_t dst = S.run[d] + (i - S.tbase[d]);
        if (!GN_CHECK(dst < n)) continue;
        kout[dst] = key;
        if (VALS) vout[dst] = sv[i];
    }
}

// Sorts of at most one tile (n <= RS_TILE) in one launch of one block: each pass ranks the
// keys by digit in shared memory (the tile's digit order is the sorted order); the next pass
// ranks a copy of that order, and the last writes it to keys_alt / vals_alt.
template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS) k_sort_tile(const uint64_t *__restrict__ keys,
                                                          uint64_t *__restrict__ keys_alt,
                                                          const uint32_t *__restrict__ vals,
                                                          uint32_t *__restrict__ vals_alt, uint32_t n, int bit_lo,
                                                          int bit_hi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RsSmem &S = *reinterpret_cast<RsSmem *>(smem_raw);
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw + ((sizeof(RsSmem) + 15) / 16) * 16);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + RS_TILE);
    uint64_t *ck = reinterpret_cast<uint64_t *>(sv + RS_TILE);  // copy of the last pass's order
    uint32_t *cv = reinterpret_cast<uint32_t *>(ck + RS_TILE);
    for (int shift = bit_lo; shift < bit_hi; shift += 8) {
        const uint32_t mask = (1u << min(8, bit_hi - shift)) - 1u;
        if (shift == bit_lo) {
            rs_rank_tile<VALS>(keys, vals, 0, n, shift, mask, S, sk, sv);
        } else {
            for (uint32_t i = threadIdx.x; i < n; i += RS_THREADS) {
                ck[i] = sk[i];
                if (VALS) cv[i] = sv[i];
            }
            __syncthreads();
            rs_rank_tile<VALS>(ck, cv, 0, n, shift, mask, S, sk, sv);
        }
    }
    for (uint32_t i = threadIdx.x; i < n; i += RS_THREADS) {
        keys_alt[i] = sk[i];
        if (VALS) vals_alt[i] = sv[i];
    }
}

static size_t rs_smem_bytes() {
    return ((sizeof(RsSmem) + 15) / 16) * 16 + (size_t)RS_TILE * (sizeof(uint64_t) + sizeof(uint32_t));
}

struct RsGeom {
    int grid;
    uint64_t chunk;
};

static RsGeom rs_geometry(uint64_t n) {
    static int occ = 0;
    if (!occ) {
        size_t smem = rs_smem_bytes();
        cudaFuncSetAttribute(k_rs_downsweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_rs_downsweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_rs_downsweep<true>, RS_THREADS, smem);
        occ = std::max(1, std::min(o, RS_MAX_GRID_PER_SM));
    }
    uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    uint64_t g = std::min<uint64_t>((uint64_t)num_sms() * occ, std::max<uint64_t>(tiles, 1));
    uint64_t tiles_per = (tiles + g - 1) / g;
    if (tiles_per == 0) tiles_per = 1;
    RsGeom geo;
    geo.chunk = tiles_per * RS_TILE;
    geo.grid = (int)std::max<uint64_t>(1, (n + geo.chunk - 1) / geo.chunk);
    return geo;
}

// Scratch of the single-pass sort: digit counts (u32) of every pass, the passes' ticket
// counters and a status word, then the tile states.
constexpr size_t OS_HIST_OFF = 0, OS_CTR_OFF = OS_MAX_PASSES * 256 * 4, OS_STATE_OFF = OS_CTR_OFF + 64;

static size_t os_scratch_bytes(uint64_t tiles) { return OS_STATE_OFF + (size_t)tiles * 256 * 8; }

size_t radix_scratch_bytes(uint64_t n) {
    size_t g = (size_t)num_sms() * RS_MAX_GRID_PER_SM;
    size_t cnt = 256 * g;
    const size_t three = cnt * sizeof(uint32_t) + (cnt + 1) * sizeof(uint64_t) + scan_scratch_bytes(cnt) + 256;
    const uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    return tiles <= OS_MAX_TILES ? std::max(three, os_scratch_bytes(tiles)) : three;
}

const RadixTag TAG_HIT_SORT{"hit_sort_hist", "hit_sort_pass", "hit_sort_upsweep", "hit_sort_downsweep"};
const RadixTag TAG_INDEX_SORT{"index_sort_hist", "index_sort_pass", "index_sort_upsweep", "index_sort_downsweep"};
const RadixTag TAG_RECORD_SORT{"record_sort_hist", "record_sort_pass", "record_sort_upsweep",
                               "record_sort_downsweep"};

thread_local KernelTimer *g_ktimer = nullptr;
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Single-pass sort (tiles <= OS_MAX_TILES): one histogram launch (first pass), then one
// launch per pass.  drop_first keeps the first tile from publishing its counts (tests of
// the bounded wait).
static bool radix_sort_onepass(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint64_t n,
                               int bit_lo, int bit_hi, void *scratch, cudaStream_t s, const RadixTag &tag,
                               uint32_t *status_word, long long budget, int drop_first) {
    const uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + OS_HIST_OFF);  // [p * 256 + digit]
    uint32_t *ctr = reinterpret_cast<uint32_t *>(base + OS_CTR_OFF);    // [p] tickets, [15] status
    unsigned long long *state = reinterpret_cast<unsigned long long *>(base + OS_STATE_OFF);
    uint32_t *status = status_word ? status_word : ctr + 15;
    GN_CUDA(cudaMemsetAsync(base, 0, OS_CTR_OFF + 64, s));
    GN_CUDA(cudaMemsetAsync(state, 0, (size_t)tiles * 256 * 8, s));
    const size_t smem = rs_smem_bytes();
    static std::once_flag attr_once;  // the pass kernels' shared memory exceeds the default 48 KB
    std::call_once(attr_once, [smem] {
        cudaFuncSetAttribute(k_os_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_os_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    auto digit_mask = [&](int shift) { return (1u << std::min(8, bit_hi - shift)) - 1u; };
    const unsigned hgrid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)num_sms() * 4));
    GN_LAUNCH(tag.up, n, s, k_os_hist<<<hgrid, RS_THREADS, 0, s>>>(keys, n, bit_lo, digit_mask(bit_lo), hist));
    bool flip = false;
    int p = 0;
    for (int shift = bit_lo; shift < bit_hi; shift += 8, ++p) {
        const uint32_t mask = digit_mask(shift);
        const int nshift = shift + 8;
        uint32_t *next = nshift < bit_hi ? hist + (p + 1) * 256 : nullptr;
        const uint32_t nmask = next ? digit_mask(nshift) : 0u;
        const uint64_t *kin = flip ? keys_alt : keys;
        uint64_t *kout = flip ? keys : keys_alt;
        const uint32_t *vin = flip ? vals_alt : vals;
        uint32_t *vout = flip ? vals : vals_alt;
        const uint64_t epoch = (uint64_t)(p + 1) << 56;
        if (vals)
            GN_LAUNCH(tag.down, n, s,
                      k_os_pass<true><<<(unsigned)tiles, RS_THREADS, smem, s>>>(
                          kin, vin, kout, vout, n, shift, mask, epoch, hist + p * 256, next, nshift, nmask, state,
                          ctr + p, status, budget, drop_first));
        else
            GN_LAUNCH(tag.down, n, s,
                      k_os_pass<false><<<(unsigned)tiles, RS_THREADS, smem, s>>>(
                          kin, nullptr, kout, nullptr, n, shift, mask, epoch, hist + p * 256, next, nshift, nmask,
                          state, ctr + p, status, budget, drop_first));
        flip = !flip;
    }
    return flip;
}

static bool radix_sort_impl(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint64_t n,
                            int bit_lo, int bit_hi, void *scratch, cudaStream_t s, const RadixTag &tag,
                            uint32_t *status_word, long long budget, int drop_first, bool three_kernel) {
    if (n <= 1 || bit_hi <= bit_lo) return false;
    if (!three_kernel && n <= RS_TILE) {  // one tile: every pass in one launch of one block
        const size_t smem = rs_smem_bytes() + (size_t)RS_TILE * (sizeof(uint64_t) + sizeof(uint32_t));
        static std::once_flag attr_once;
        std::call_once(attr_once, [smem] {
            cudaFuncSetAttribute(k_sort_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(k_sort_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (vals)
            GN_LAUNCH(tag.down, n, s,
                      k_sort_tile<true><<<1, RS_THREADS, smem, s>>>(keys, keys_alt, vals, vals_alt, (uint32_t)n, bit_lo,
                                                                     bit_hi));
        else
            GN_LAUNCH(tag.down, n, s,
                      k_sort_tile<false><<<1, RS_THREADS, smem, s>>>(keys, keys_alt, nullptr, nullptr, (uint32_t)n,
                                                                      bit_lo, bit_hi));
        return true;  // the sorted keys are in keys_alt
    }
    if (!three_kernel && (n + RS_TILE - 1) / RS_TILE <= OS_MAX_TILES && bit_hi - bit_lo <= 8 * OS_MAX_PASSES)
        return radix_sort_onepass(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, scratch, s, tag, status_word,
                                  budget, drop_first);
    RsGeom geo = rs_geometry(n);
    size_t cnt = (size_t)256 * geo.grid;
    uint32_t *counts = static_cast<uint32_t *>(scratch);
    uint64_t *offs = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(counts + cnt) + 15) & ~(uintptr_t)15);
    void *scan_scratch = reinterpret_cast<void *>(
        (reinterpret_cast<uintptr_t>(offs + cnt + 1) + 15) & ~(uintptr_t)15);
    const size_t smem = rs_smem_bytes();
    bool flip = false;
    for (int shift = bit_lo; shift < bit_hi; shift += 8) {
        int nbits = std::min(8, bit_hi - shift);
        uint32_t mask = (1u << nbits) - 1u;
        const uint64_t *kin = flip ? keys_alt : keys;
        uint64_t *kout = flip ? keys : keys_alt;
        const uint32_t *vin = flip ? vals_alt : vals;
        uint32_t *vout = flip ? vals : vals_alt;
        GN_LAUNCH(tag.up3, n, s,
                  k_rs_upsweep<<<geo.grid, RS_THREADS, 0, s>>>(kin, n, geo.chunk, shift, mask, counts));
        exclusive_scan_u32(counts, offs, cnt, scan_scratch, s);
        if (vals) {
            GN_LAUNCH(tag.down3, n, s,
                      k_rs_downsweep<true><<<geo.grid, RS_THREADS, smem, s>>>(kin, vin, kout, vout, n, geo.chunk,
                                                                              shift, mask, offs));
        } else {
            GN_LAUNCH(tag.down3, n, s,
                      k_rs_downsweep<false><<<geo.grid, RS_THREADS, smem, s>>>(kin, nullptr, kout, nullptr, n,
                                                                               geo.chunk, shift, mask, offs));
        }
        flip = !flip;
    }
    return flip;
}

bool radix_sort(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint64_t n, int bit_lo,
                int bit_hi, void *scratch, cudaStream_t s, const RadixTag &tag) {
    const bool three = getenv("GN_SORT_THREE_KERNEL") != nullptr;
    return radix_sort_impl(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, scratch, s, tag, g_wait_status,
                           SCAN_WAIT_BUDGET, 0, three);
}

// Sort of caller buffers in place (keys, and vals if given) by bits [bit_lo, bit_hi) with a
// given wait budget; drop_first as in radix_sort_onepass, three_kernel forces the
// three-kernel passes.  Returns whether a wait ran out.
bool debug_sort(uint64_t *keys, uint32_t *vals, uint64_t n, int bit_lo, int bit_hi, long long budget,
                int drop_first, bool three_kernel, cudaStream_t s) {
    DeviceArena arena(s);
    uint64_t *keys_alt = arena.alloc_n<uint64_t>(std::max<uint64_t>(n, 1));
    uint32_t *vals_alt = vals ? arena.alloc_n<uint32_t>(std::max<uint64_t>(n, 1)) : nullptr;
    void *scr = arena.alloc(radix_scratch_bytes(n));
    uint32_t *st = arena.alloc_n<uint32_t>(1);
    GN_CUDA(cudaMemsetAsync(st, 0, 4, s));
    const bool flip = radix_sort_impl(keys, keys_alt, vals, vals_alt, n, bit_lo, bit_hi, scr, s, TAG_RECORD_SORT, st,
                                      budget, drop_first, three_kernel);
    if (flip) {
        GN_CUDA(cudaMemcpyAsync(keys, keys_alt, 8 * n, cudaMemcpyDeviceToDevice, s));
        if (vals) GN_CUDA(cudaMemcpyAsync(vals, vals_alt, 4 * n, cudaMemcpyDeviceToDevice, s));
    }
    uint32_t h = 0;
    GN_CUDA(cudaMemcpyAsync(&h, st, 4, cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    return (h & DEV_ERR_TIMEOUT) != 0;
}

// --------------------------------------------------------- record sort --
struct KeyFields {
    int n;
    int word[4];
    int shift[4];
    uint32_t mask[4];
    int desc[4];
};

__global__ void k_iota(uint32_t *p, uint32_t n) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// keys[i] from the fields of record perm[i]; with first set, perm is the identity and is
// written here (perm[i] = i).
__global__ void k_make_keys(const uint32_t *__restrict__ recs, int rec_words, uint32_t *__restrict__ perm,
                            uint32_t n, KeyFields f, uint64_t *__restrict__ keys, int first) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t pi = i;
    if (first) perm[i] = i;
    else pi = perm[i];
    const uint32_t *r = recs + (uint64_t)pi * rec_words;
    uint64_t k = 0;
    for (int j = 0; j < f.n; ++j) {
        uint32_t v = r[f.word[j]];
        if (f.desc[j]) v = ~v;
        k |= (uint64_t)(v & f.mask[j]) << f.shift[j];
    }
    keys[i] = k;
}

void sort_records(const uint32_t *recs, int rec_words, uint32_t n, const std::vector<SortField> &fields,
                  uint32_t *perm_out, DeviceArena &arena, cudaStream_t s) {
    if (n == 0) return;
    unsigned grid = (n + 255) / 256;
    uint32_t *perm = perm_out;
    uint32_t *perm_alt = arena.alloc_n<uint32_t>(n);
    uint64_t *keys = arena.alloc_n<uint64_t>(n);
    uint64_t *keys_alt = arena.alloc_n<uint64_t>(n);
    void *scratch = arena.alloc(radix_scratch_bytes(n));
    // group fields into <= 64-bit keys, least significant group first (the first group's key
    // launch also writes the identity permutation)
    bool first = true;
    int fi = (int)fields.size() - 1;
    while (fi >= 0) {
        KeyFields kf;
        kf.n = 0;
        int used = 0;
        while (fi >= 0 && kf.n < 4 && used + fields[fi].bits <= 64) {
            const SortField &sf = fields[fi];
            kf.word[kf.n] = sf.word;
            kf.shift[kf.n] = used;
            kf.mask[kf.n] = sf.bits >= 32 ? 0xFFFFFFFFu : ((1u << sf.bits) - 1u);
            kf.desc[kf.n] = sf.desc ? 1 : 0;
            used += sf.bits;
            ++kf.n;
            --fi;
        }
        if (kf.n == 0) throw Error{GN_EINTERNAL, "sort field wider than 64 bits"};
        if (used == 0) continue;
        GN_LAUNCH("k_make_keys", n, s,
                  k_make_keys<<<grid, 256, 0, s>>>(recs, rec_words, perm, n, kf, keys, first ? 1 : 0));
        first = false;
        bool flipped = radix_sort(keys, keys_alt, perm, perm_alt, n, 0, used, scratch, s, TAG_RECORD_SORT);
        if (flipped) std::swap(perm, perm_alt);
    }
    if (first) GN_LAUNCH("k_iota", n, s, k_iota<<<grid, 256, 0, s>>>(perm, n));  // no field has bits
    if (perm != perm_out) GN_CUDA(cudaMemcpyAsync(perm_out, perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
}

__global__ void k_gather_records(const uint32_t *__restrict__ in, int W, const uint32_t *__restrict__ perm,
                                 uint32_t n, uint32_t *__restrict__ out) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * W) return;
    uint32_t i = (uint32_t)(t / W), w = (uint32_t)(t % W);
    out[t] = in[(uint64_t)perm[i] * W + w];
}

void gather_records(const uint32_t *in, int rec_words, const uint32_t *perm, uint32_t n, uint32_t *out,
                    cudaStream_t s) {
    if (n == 0) return;
    uint64_t tot = (uint64_t)n * rec_words;
    GN_LAUNCH("k_gather_records", n, s,
              k_gather_records<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(in, rec_words, perm, n, out));
}

}  // namespace gn
