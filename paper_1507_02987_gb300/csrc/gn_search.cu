// gn_search.cu - the search phases of the paper ("Searching process" section) on
// the device, for a batch of independent queries:
//   a5  input processing: rolling k-mer code of every query offset
//   a6  index lookup: gather of every occurrence of every code (hits)
//   a7  grouping: radix sort of hits by (diagonal key, query, query offset)
//   a8  merging of hits at most D apart on one (sequence, diagonal) into HSPs
//   a9  X-drop ungapped extension of both HSP ends
//   a10 merging of overlapped HSPs (single sweep per query and sequence)
//   a11 selection of the longest HSPs per query
//   a12 banded affine-gap Smith-Waterman of each selected HSP
//   a13 ranking by score, duplicate removal, e-value and bit score
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "gn_internal.cuh"

namespace gn {

// HSP record (7 words, same layout as gn_hsp)
struct DevHsp {
    uint32_t qi, seq, qs, qe, ds, de, len;
};
static_assert(sizeof(DevHsp) == 28, "DevHsp layout");
constexpr int HSP_WORDS = 7;
enum { W_QI = 0, W_SEQ = 1, W_QS = 2, W_QE = 3, W_DS = 4, W_DE = 5, W_LEN = 6 };

// alignment record (8 words)
struct DevAln {
    uint32_t qi, seq, qs, qe, ds, de;
    int32_t score;
    uint32_t pad;
};
static_assert(sizeof(DevAln) == 32, "DevAln layout");
constexpr int ALN_WORDS = 8;
enum { A_QI = 0, A_SEQ = 1, A_QS = 2, A_QE = 3, A_DS = 4, A_DE = 5, A_SCORE = 6 };

// ------------------------------------------------------ a5: query codes --
// Per global query offset x: query id and offset (qinfo = qi << 16 | qpos),
// k-mer code and the length of its occurrence list (0 for no window).
__global__ void k_query_codes(const uint64_t *__restrict__ qstart, uint32_t nq, uint64_t M,
                              const uint32_t *__restrict__ qpk, const uint32_t *__restrict__ qnb, SeedShape sh,
                              const uint64_t *__restrict__ off, uint32_t *__restrict__ codes,
                              uint32_t *__restrict__ qinfo, uint32_t *__restrict__ cnt,
                              uint32_t *__restrict__ src) {
    uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= M) return;
    uint32_t qi = dev_upper_index(qstart, nq + 1, x);
    uint64_t qpos = x - qstart[qi];
    uint64_t m = qstart[qi + 1] - qstart[qi];
    uint32_t c = 0, n = 0;
    uint64_t o = 0;
    if (qpos + (uint64_t)sh.span <= m && !dev_seed_has_nonbase(qnb, x, sh)) {
        c = dev_seed_code(qpk, x, sh);
        o = off[c];
        n = (uint32_t)(off[c + 1] - o);
    }
    codes[x] = c;
    qinfo[x] = (qi << 16) | (uint32_t)qpos;
    cnt[x] = n;
    src[x] = (uint32_t)o;  // occurrence indices fit 32 bits: the bank holds < 2^32 bases
}

// Seed hits of each query of a batch (request admission): one block per query sums the
// occurrence-list lengths of the seed codes of its offsets, read from ASCII bases.
__device__ __forceinline__ uint32_t ascii_base_code(uint8_t b) {
    const uint32_t c = b & 0xDFu;
    return c == 'A' ? 0u : c == 'C' ? 1u : c == 'G' ? 2u : (c == 'T' || c == 'U') ? 3u : 4u;
}

__global__ void __launch_bounds__(256) k_request_hits(const uint8_t *__restrict__ bases,
                                                      const uint64_t *__restrict__ start, uint32_t n, SeedShape sh,
                                                      const uint64_t *__restrict__ off,
                                                      unsigned long long *__restrict__ hits) {
    __shared__ unsigned long long part[8];
    for (uint32_t q = blockIdx.x; q < n; q += gridDim.x) {
        const uint64_t b0 = start[q], m = start[q + 1] - b0;
        unsigned long long sum = 0;
        for (uint64_t x = threadIdx.x; x + (uint64_t)sh.span <= m; x += blockDim.x) {
            uint32_t code = 0;
            bool ok = true;
            for (int p = 0; p < sh.span; ++p) {
                if (!((sh.keep >> p) & 1u)) continue;
                const uint32_t c = ascii_base_code(bases[b0 + x + p]);
                ok = ok && c < 4u;
                code = (code << 2) | (c & 3u);
            }
            if (ok) sum += off[code + 1] - off[code];
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            hits[q] = t;
        }
        __syncthreads();
    }
}

void count_request_hits(const gn_index *ix, const uint8_t *bases, const uint64_t *start, uint32_t n,
                        unsigned long long *hits, cudaStream_t s) {
    if (!n) return;
    GN_LAUNCH("k_request_hits", n, s,
              k_request_hits<<<(unsigned)std::min<uint32_t>(n, (uint32_t)num_sms() * 8), 256, 0, s>>>(
                  bases, start, n, seed_shape(ix), ix->off_d, hits));
}

__global__ void k_gather_u64(const uint64_t *__restrict__ src, const uint64_t *__restrict__ idx, uint32_t n,
                             uint64_t *__restrict__ out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = src[idx[i]];
}

// ------------------------------------------------------- a6: seed gather --
// A warp takes 32 consecutive query offsets; their occurrence lists are
// copied one after another by the whole warp (coalesced reads of the list,
// coalesced writes of the hit keys).
// key = (gpos - qpos + QBIAS) << (16 + qbits) | (qi - qa) << 16 | qpos
__global__ void __launch_bounds__(256) k_seed_gather(const uint32_t *__restrict__ codes,
                                                     const uint32_t *__restrict__ qinfo,
                                                     const uint64_t *__restrict__ hoff, uint64_t xa, uint64_t xb,
                                                     uint64_t ha, const uint64_t *__restrict__ off,
                                                     const uint32_t *__restrict__ post, uint32_t qa, int qbits,
                                                     uint64_t *__restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (uint64_t x0 = xa + warp * 32; x0 < xb; x0 += nwarps * 32) {
        uint64_t x = x0 + lane;
        uint32_t my_cnt = 0;
        uint64_t my_src = 0, my_dst = 0, my_pref = 0;
        uint32_t my_qpos = 0;
        if (x < xb) {
            my_cnt = (uint32_t)(hoff[x + 1] - hoff[x]);
            if (my_cnt) {
                uint32_t qinf = qinfo[x];
                my_src = off[codes[x]];
                my_dst = hoff[x] - ha;
                my_qpos = qinf & 0xFFFFu;
                my_pref = ((uint64_t)((qinf >> 16) - qa) << 16) | my_qpos;
            }
        }
        uint32_t todo = __ballot_sync(0xffffffffu, my_cnt != 0);
        while (todo) {
            int src = __ffs(todo) - 1;
            todo &= todo - 1;
            uint32_t cnt = __shfl_sync(0xffffffffu, my_cnt, src);
            uint64_t sp = __shfl_sync(0xffffffffu, my_src, src);
            uint64_t dp = __shfl_sync(0xffffffffu, my_dst, src);
            uint64_t pref = __shfl_sync(0xffffffffu, my_pref, src);
            uint32_t qpos = __shfl_sync(0xffffffffu, my_qpos, src);
            for (uint32_t j = lane; j < cnt; j += 32) {
                uint64_t g = post[sp + j];
                uint64_t gkey = g + QBIAS - qpos;
                keys[dp + j] = (gkey << (16 + qbits)) | pref;
            }
        }
    }
}

// ------------------------------------------------------ a8: hit merging --
struct HitKey {
    uint64_t gkey;  // gpos - qpos + QBIAS
    uint32_t ql, qpos;
};

__device__ __forceinline__ HitKey dec_key(uint64_t key, int qbits) {
    HitKey h;
    h.qpos = (uint32_t)(key & 0xFFFFu);
    h.ql = (uint32_t)((key >> 16) & ((1ull << qbits) - 1ull));
    h.gkey = key >> (16 + qbits);
    return h;
}

// Chains of sorted hit keys: a hit starts a chain unless the previous key has the same
// diagonal and query, lies at most D query offsets before it and in the same bank
// sequence; the head walks its chain, whose hits must end before its sequence does.
__global__ void k_hit_merge(const uint64_t *__restrict__ keys, uint64_t n, int qbits, uint32_t qa, int k,
                            uint32_t D, uint32_t min_len, SeqMap sm, DevHsp *__restrict__ out,
                            uint32_t *__restrict__ count, uint32_t cap, uint32_t *__restrict__ status) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t key = keys[i];
        const HitKey a = dec_key(key, qbits);
        const uint64_t gpos = a.gkey - QBIAS + a.qpos;
        const uint32_t sq = dev_seq_of(sm, gpos);
        if (i > 0) {
            const uint64_t prev = keys[i - 1];
            const uint32_t qp = (uint32_t)(prev & 0xFFFFu);
            if ((prev >> 16) == (key >> 16) && a.qpos - qp <= D && sm.start[sq] <= gpos - (a.qpos - qp)) continue;
        }
        const uint64_t seq_end = sm.start[sq + 1];
        uint64_t j = i, kj = key;
        while (j + 1 < n) {
            const uint64_t kn = keys[j + 1];
            const uint32_t qn = (uint32_t)(kn & 0xFFFFu);
            if ((kn >> 16) != (key >> 16) || qn - (uint32_t)(kj & 0xFFFFu) > D || a.gkey - QBIAS + qn >= seq_end) break;
            kj = kn;
            ++j;
        }
        const uint32_t qs = a.qpos, qe = (uint32_t)(kj & 0xFFFFu) + (uint32_t)k;
        const uint32_t len = qe - qs;
        if (len < min_len) continue;
        const uint32_t ds = (uint32_t)(gpos - sm.start[sq]);
        const uint32_t slot = atomicAdd(count, 1u);
        if (slot < cap) {
            DevHsp h;
            h.qi = qa + a.ql; h.seq = sq; h.qs = qs; h.qe = qe; h.ds = ds; h.de = ds + len; h.len = len;
            out[slot] = h;
        } else {
            atomicOr(status, DEV_ERR_CAPACITY);
        }
    }
}

// ------------------------------------------ a6-a8: bucketed hit grouping --
// Hits of query i are partitioned into 2^b_i buckets by the high bits of their
// diagonal key G' = gpos - qpos + QBIAS (bucket = bbase[i] + (G' >> bshift[i])).
// Every (query, diagonal) lies in one bucket, so each bucket is grouped on its
// own.  A diagonal holding a single hit cannot form an HSP when min_hsp_len > k,
// so such hits are dropped before the (small) sort by (G', qpos) that the
// chaining needs.  Bucket entry: G' << 16 | qpos.

// Tile-level bucketing: a CTA takes tpos consecutive query offsets (the core).
// With the repeat filter on (min_hsp_len > k and D <= BT_MAX_D), every hit of the
// core and of the D offsets on either side (the halo) is first entered, by its
// (query, diagonal), into a shared-memory Bloom filter "seen" (three bits of one
// 32-bit word per key); a hit that finds all its bits set already enters its key
// into a second one, "seen twice" (two bits of one word).  A core hit can only be
// part of a chain of two or more hits if another hit lies on its diagonal within D
// query offsets, and all those offsets are inside core + halo; the later of two
// hits with one key always finds that key's "seen" bits set.  A Bloom filter has
// no false negatives, so a core hit whose "seen twice" bits are not all set cannot
// reach min_hsp_len and is dropped here; a false positive only keeps an extra hit.
constexpr int BT_MAX_D = 256;  // largest hit distance the tile filter supports

// The tile's occurrence lists are read in aligned quads of four entries (16-byte
// loads): the list of offset i, occurrences [beg_i, end_i), covers quads beg_i / 4
// to (end_i - 1) / 4 of the occurrence array, and the quads of all the tile's lists
// form one index space.  Warps take chunks of BF_QCHUNK quads from a shared counter
// (lane l holds quads c * BF_QCHUNK + 32 v + l, v < BF_QV), whatever lists they fall
// in, so every lane has work and a long list is shared by many warps.  A quad lies
// in one list; entries of a neighbouring list that share its 16 bytes are masked.
constexpr int BF_QV = 2;
constexpr int BF_QCHUNK = 32 * BF_QV;
constexpr int BF_CMAX = 512;  // chunks whose first list is tabulated (later ones are searched)
// Kept hits of a tile are staged in shared memory (stage_cap of them, the room the
// launch leaves) and placed in their buckets after the tile's placement pass, all
// threads at once, so that their global atomics overlap instead of stalling each warp's
// pass; hits past the stage's room are placed directly.
constexpr int BF_STAGE_BYTES = 14;  // per staged hit: key, bucket, query

// Key of a hit for the filters: the low 32 bits of its diagonal key G' mixed with its
// query (kadd = QBIAS - query offset, kx = query in chunk times an odd constant).
__device__ __forceinline__ uint32_t bf_key(uint32_t ent, uint32_t kadd, uint32_t kx) { return (ent + kadd) ^ kx; }
// Positions of a key in the two filters: the word of each from the top bits of one
// multiplicative (Fibonacci) hash, which spreads the keys of nearby diagonals over the
// words; the bits inside the word from 5-bit fields of the key itself, which differ
// between nearby diagonals.
__device__ __forceinline__ uint32_t bf_hash(uint32_t key) { return key * 0x9E3779B1u; }
// 1 << (x mod 32) in one funnel shift (the shift amount wraps modulo 32)
__device__ __forceinline__ uint32_t bit_of(uint32_t x) { return __funnelshift_l(0u, 1u, x); }
__device__ __forceinline__ uint32_t bf_mask(uint32_t key) {  // "seen": three bits
    return bit_of(key) | bit_of(key >> 5) | bit_of(key >> 10);
}
__device__ __forceinline__ uint32_t bf2_mask(uint32_t key) {  // "seen twice": two bits
    return bit_of(key >> 15) | bit_of(key >> 20);
}

// Shared-memory table of a tile's query offsets lo + i, i in [0, span): quad prefix
// relative to the tile's first quad (span + 1 entries), occurrence range [beg, end),
// (query in chunk << 16 | query offset), and the query's bucket base and shift;
// cs[c] is the offset holding quad c * BF_QCHUNK for the first BF_CMAX chunks.
// Tile-relative quad indices fit 32 bits: a query chunk holds < 2^32 hits.
struct TileTable {
    uint32_t *qp, *beg, *end, *qq, *bb, *cs;
    uint8_t *bs;
    uint32_t span, nchunks;
    uint64_t nquads;  // quads of the occurrence array (checked builds)
};

// Last table index i in [i_lo, i_hi] with qp[i] <= e: the offset whose list holds quad e.
__device__ __forceinline__ uint32_t tile_find(const uint32_t *qp, uint32_t i_lo, uint32_t i_hi, uint32_t e) {
    while (i_lo < i_hi) {
        const uint32_t mid = (i_lo + i_hi + 1) >> 1;
        if (qp[mid] <= e) i_lo = mid;
        else i_hi = mid - 1;
    }
    return i_lo;
}

__device__ __forceinline__ uint32_t tile_chunk_list(const TileTable &t, uint32_t c) {
    return c < BF_CMAX ? t.cs[c] : tile_find(t.qp, 0, t.span - 1, c * BF_QCHUNK);
}

// The BF_QV quads a lane holds of one chunk: entries (loads in flight until used),
// table index, occurrence index of the first entry, and whether the quad is inside
// the pass's quad range.
struct QuadLoad {
    uint4 ent[BF_QV];
    uint32_t idx[BF_QV], occ[BF_QV];
    bool ok[BF_QV];
};

// Issues the loads of chunk c, masked to the quad range [r0, r1): one search per lane
// for its first quad's list, then a boundary check per quad.
__device__ __forceinline__ void tile_quad_load(const TileTable &t, uint32_t c, uint32_t r0, uint32_t r1,
                                               const uint4 *__restrict__ post4, QuadLoad &L) {
    const int lane = threadIdx.x & 31;
    const uint32_t e0 = c * BF_QCHUNK + lane;
    const uint32_t i0 = tile_chunk_list(t, c);
    const uint32_t i1 = c + 1 < t.nchunks ? tile_chunk_list(t, c + 1) : t.span - 1;
    uint32_t i = tile_find(t.qp, i0, i1, e0);
    uint32_t nx = t.qp[i + 1];
#pragma unroll
    for (int v = 0; v < BF_QV; ++v) {
        const uint32_t e = e0 + 32u * v;
        while (e >= nx && i < i1) {  // the next non-empty list
            ++i;
            nx = t.qp[i + 1];
        }
        L.idx[v] = i;
        L.ok[v] = e >= r0 && e < r1;
        const uint32_t q = (t.beg[i] >> 2) + (e - t.qp[i]);
        L.occ[v] = q << 2;
        if (L.ok[v] && !GN_CHECK(q < t.nquads)) L.ok[v] = false;
        L.ent[v] = L.ok[v] ? __ldg(&post4[q]) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Calls f(L) for every chunk of quads meeting [r0, r1) (tile-relative quad indices);
// all lanes of a warp call f together.  A warp issues the loads of its next chunk
// before it processes the current one.
template <class F>
__device__ __forceinline__ void for_tile_quads(const TileTable &t, uint32_t r0, uint32_t r1, uint32_t *ctr,
                                               const uint4 *__restrict__ post4, F &&f) {
    const int lane = threadIdx.x & 31;
    if (r0 >= r1) return;
    const uint32_t c0 = r0 / BF_QCHUNK, nc = (r1 + BF_QCHUNK - 1) / BF_QCHUNK - c0;
    auto claim = [&]() {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(ctr, 1u);
        return __shfl_sync(0xffffffffu, c, 0);
    };
    uint32_t c = claim();
    if (c >= nc) return;
    QuadLoad cur, nxt;
    tile_quad_load(t, c0 + c, r0, r1, post4, cur);
    for (;;) {
        const uint32_t cn = claim();
        const bool more = cn < nc;
        if (more) tile_quad_load(t, c0 + cn, r0, r1, post4, nxt);
        f(cur);
        if (!more) break;
        cur = nxt;
    }
}

__device__ __forceinline__ uint32_t quad_word(const uint4 &q, int u) {
    return u == 0 ? q.x : u == 1 ? q.y : u == 2 ? q.z : q.w;
}

// Exclusive scan of one value per thread over the block (blockDim.x a multiple of 32,
// at most 1,024); wtot holds 32 words of shared memory.
__device__ __forceinline__ uint32_t bf_block_scan(uint32_t v, uint32_t *wtot, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? wtot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wtot[lane] = w;
    }
    __syncthreads();
    total = wtot[nw - 1];
    const uint32_t before = warp ? wtot[warp - 1] : 0u;
    __syncthreads();  // wtot is reused by the next call
    return before + x - v;
}

// Places one kept hit (key = G' << 16 | query offset, ql = query in chunk) in bucket b:
// a global atomic reserves its slot; past the bucket's capacity it goes to the spill
// list in global hit-key format.
__device__ __forceinline__ void bucket_place(uint32_t b, uint64_t key, uint32_t ql, uint32_t *__restrict__ bcount,
                                             uint64_t *__restrict__ bkeys, uint32_t bcap, uint64_t *__restrict__ spill,
                                             unsigned long long *__restrict__ spill_count,
                                             unsigned long long spill_cap, int qbits, uint32_t NB) {
    if (!GN_CHECK(b < NB)) return;
    const uint32_t slot = atomicAdd(&bcount[b], 1u);
    if (slot < bcap) {
        bkeys[(uint64_t)b * bcap + slot] = key;
    } else {
        const unsigned long long at = atomicAdd(spill_count, 1ull);
        if (at < spill_cap) spill[at] = ((key >> 16) << (16 + qbits)) | ((uint64_t)ql << 16) | (key & 0xFFFFu);
    }
}

// Bucket fill: one kernel per query chunk.  Each tile (tpos core offsets) enters the
// hits of core + halo into the "seen" / "seen twice" filters (repeat filter), then
// places every kept core hit: one global atomic reserves its slot in its bucket.
// Buckets have a fixed capacity bcap; hits past it go to the spill list in global
// hit-key format, which the global sort path handles.  count_only: no placement,
// kept_total[0] counts the kept core hits and kept_total[1] all core hits of the
// tiles visited (tiles 0, tile_step, 2 tile_step, ...).  kept_total[2] hands out the
// tiles (zero at launch).
// FB, FB2: the filters' sizes in bits as constants (0: the run-time fbits, fbits2).
template <int FB, int FB2>
__global__ void __launch_bounds__(512, 2) k_bucket_fill(
    const uint32_t *__restrict__ qinfo, const uint32_t *__restrict__ src, const uint64_t *__restrict__ hoff,
    uint64_t xa, uint64_t xb, const uint32_t *__restrict__ post, uint32_t qa, const uint32_t *__restrict__ bbase,
    const uint32_t *__restrict__ bshift, uint32_t *__restrict__ bcount, uint64_t *__restrict__ bkeys, uint32_t bcap,
    uint64_t *__restrict__ spill, unsigned long long *__restrict__ spill_count, unsigned long long spill_cap,
    int qbits, int filter, uint32_t D, int tpos, int fbits, int fbits2, unsigned long long *__restrict__ kept_total,
    uint32_t tile_step, int count_only, uint32_t stage_cap, uint32_t NB, uint64_t post_quads) {
    extern __shared__ __align__(16) unsigned char bf_smem[];
    const uint32_t halo = filter ? D : 0u;
    const uint32_t span_max = (uint32_t)tpos + 2u * halo;
    const int wbits = (FB ? FB : fbits) - 5, wbits2 = (FB2 ? FB2 : fbits2) - 5;
    const uint32_t nwords = filter ? 1u << wbits : 0u, nwords2 = filter ? 1u << wbits2 : 0u;
    const uint4 *__restrict__ post4 = reinterpret_cast<const uint4 *>(post);
    uint64_t *stage_key = reinterpret_cast<uint64_t *>(bf_smem);  // G' << 16 | query offset
    uint32_t *seen = reinterpret_cast<uint32_t *>(stage_key + stage_cap);
    uint32_t *seen2 = seen + nwords;
    TileTable t;
    t.nquads = post_quads;
    t.qp = seen2 + nwords2;
    t.beg = t.qp + span_max + 1;
    t.end = t.beg + span_max;
    t.qq = t.end + span_max;
    t.bb = t.qq + span_max;
    t.cs = t.bb + span_max;
    uint32_t *stage_b = t.cs + BF_CMAX;                                 // bucket
    uint16_t *stage_q = reinterpret_cast<uint16_t *>(stage_b + stage_cap);  // query in chunk
    t.bs = reinterpret_cast<uint8_t *>(stage_q + stage_cap);
    __shared__ uint32_t ctr, nstage;
    __shared__ uint32_t wtot[32];
    uint32_t my_kept = 0;
    unsigned long long my_core = 0;  // core hits of the visited tiles (count-only runs)
    // tiles from a counter (kept_total[2]): blocks that drew small tiles take more
    __shared__ uint64_t s_t0;
    for (;;) {
        if (threadIdx.x == 0) s_t0 = xa + atomicAdd(kept_total + 2, 1ull) * tile_step * (uint64_t)tpos;
        __syncthreads();
        const uint64_t t0 = s_t0;
        if (t0 >= xb) break;
        const uint64_t t1 = min(xb, t0 + (uint64_t)tpos);
        const uint64_t lo = t0 - xa > halo ? t0 - halo : xa, hi = min(xb, t1 + halo);
        const uint32_t span = (uint32_t)(hi - lo);
        // per-offset table; quad counts first, then their exclusive scan in place
        for (uint32_t i = threadIdx.x; i < span; i += blockDim.x) {
            const uint64_t x = lo + i;
            const uint32_t b = src[x], n = (uint32_t)(hoff[x + 1] - hoff[x]);
            t.beg[i] = b;
            t.end[i] = b + n;
            t.qp[i] = n ? ((b + n + 3u) >> 2) - (b >> 2) : 0u;
            const uint32_t qinf = qinfo[x];
            const uint32_t ql = (qinf >> 16) - qa;
            t.qq[i] = (ql << 16) | (qinf & 0xFFFFu);
            t.bb[i] = bbase[ql];
            t.bs[i] = (uint8_t)bshift[ql];
        }
        for (uint32_t i = threadIdx.x; i < nwords + nwords2; i += blockDim.x) seen[i] = 0u;
        if (threadIdx.x == 0) ctr = nstage = 0;
        if (count_only && threadIdx.x == 0) my_core += hoff[t1] - hoff[t0];
        __syncthreads();
        {
            const uint32_t per = (span + blockDim.x - 1) / blockDim.x;
            const uint32_t a = min(span, threadIdx.x * per), b = min(span, a + per);
            uint32_t sum = 0;
            for (uint32_t i = a; i < b; ++i) sum += t.qp[i];
            uint32_t total = 0;
            uint32_t run = bf_block_scan(sum, wtot, total);
            for (uint32_t i = a; i < b; ++i) {
                const uint32_t nq = t.qp[i];
                t.qp[i] = run;
                run += nq;
            }
            if (threadIdx.x == 0) t.qp[span] = total;
        }
        __syncthreads();
        t.span = span;
        t.nchunks = (t.qp[span] + BF_QCHUNK - 1) / BF_QCHUNK;
        // chunk -> offset of its first quad
        for (uint32_t i = threadIdx.x; i < span; i += blockDim.x) {
            const uint32_t ca = (t.qp[i] + BF_QCHUNK - 1) / BF_QCHUNK;
            const uint32_t cb = min((t.qp[i + 1] + BF_QCHUNK - 1) / BF_QCHUNK, (uint32_t)BF_CMAX);
            for (uint32_t c = ca; c < cb; ++c) t.cs[c] = i;
        }
        __syncthreads();
        if (filter) {
            for_tile_quads(t, 0, t.qp[span], &ctr, post4, [&](const QuadLoad &L) {
#pragma unroll
                for (int v = 0; v < BF_QV; ++v) {
                    if (!L.ok[v]) continue;
                    const uint32_t qq = t.qq[L.idx[v]];
                    const uint32_t kadd = QBIAS - (qq & 0xFFFFu), kx = (qq >> 16) * 0x85EBCA77u;
                    // entries of a neighbouring list that share the quad are entered too: an
                    // extra key can only add false positives
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t key = bf_key(quad_word(L.ent[v], u), kadd, kx);
                        const uint32_t h = bf_hash(key), m = bf_mask(key);
                        const uint32_t old = atomicOr(&seen[h >> (32 - wbits)], m);
                        if ((old & m) == m) atomicOr(&seen2[h >> (32 - wbits2)], bf2_mask(key));
                    }
                }
            });
            __syncthreads();
            if (threadIdx.x == 0) ctr = 0;
            __syncthreads();
        }
        // place the kept core hits (count them only, when sampling the keep rate)
        for_tile_quads(t, t.qp[t0 - lo], t.qp[t1 - lo], &ctr, post4, [&](const QuadLoad &L) {
#pragma unroll
            for (int v = 0; v < BF_QV; ++v) {
                if (!L.ok[v]) continue;
                const uint32_t i = L.idx[v], qq = t.qq[i], beg = t.beg[i], end = t.end[i], occ = L.occ[v];
                // entries of this list in the quad: from beg - occ (first quad) to end - occ (last)
                const uint32_t first = occ < beg ? beg - occ : 0u, last = end - occ < 4u ? end - occ : 4u;
                uint32_t keep = (0xFu >> (4u - last)) & (0xFu << first);  // bit u: entry u is a kept hit
                if (filter) {
                    const uint32_t kadd = QBIAS - (qq & 0xFFFFu), kx = (qq >> 16) * 0x85EBCA77u;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t key = bf_key(quad_word(L.ent[v], u), kadd, kx);
                        const uint32_t m2 = bf2_mask(key);
                        if ((seen2[bf_hash(key) >> (32 - wbits2)] & m2) != m2) keep &= ~(1u << u);
                    }
                }
                if (!keep) continue;
                my_kept += __popc(keep);
                if (count_only) continue;
                const uint32_t bb = t.bb[i], bs = t.bs[i];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!(keep >> u & 1u)) continue;
                    const uint64_t gk = (uint64_t)quad_word(L.ent[v], u) + QBIAS - (qq & 0xFFFFu);
                    const uint32_t b = bb + (uint32_t)(gk >> bs);
                    const uint64_t key = (gk << 16) | (qq & 0xFFFFu);
                    const uint32_t at = atomicAdd(&nstage, 1u);
                    if (at < stage_cap) {
                        stage_key[at] = key;
                        stage_b[at] = b;
                        stage_q[at] = (uint16_t)(qq >> 16);
                    } else {
                        bucket_place(b, key, qq >> 16, bcount, bkeys, bcap, spill, spill_count, spill_cap, qbits,
                                     NB);
                    }
                }
            }
        });
        if (!count_only) {
            __syncthreads();
            const uint32_t ns = min(nstage, stage_cap);
            for (uint32_t j = threadIdx.x; j < ns; j += blockDim.x)
                bucket_place(stage_b[j], stage_key[j], stage_q[j], bcount, bkeys, bcap, spill, spill_count, spill_cap,
                             qbits, NB);
        }
        __syncthreads();  // the table and filters are rebuilt for the next tile
    }
    if (my_kept) atomicAdd(kept_total, (unsigned long long)my_kept);
    if (my_core) atomicAdd(kept_total + 1, my_core);
}

// Dynamic shared memory of k_bucket_fill: staged kept hits, filters, offset table.
static size_t bucket_fill_smem(int tpos, uint32_t halo, int filter, int fbits, int fbits2, uint32_t stage_cap) {
    const size_t span_max = (size_t)tpos + 2 * halo;
    return (size_t)stage_cap * BF_STAGE_BYTES + (filter ? ((1u << fbits) + (1u << fbits2)) / 8 : 0) +
           (span_max + 1) * 4 + span_max * 17 + 4 * BF_CMAX;
}

__global__ void k_bucket_query(const uint32_t *__restrict__ bbase, uint32_t nqc, uint32_t NB,
                               uint16_t *__restrict__ bq) {
    uint32_t q = blockIdx.x;
    if (q >= nqc) return;
    for (uint32_t b = bbase[q] + threadIdx.x; b < bbase[q + 1]; b += blockDim.x) bq[b] = (uint16_t)q;
}

// Chains of candidates sorted by (G', qpos) within one bucket (one query): candidate i
// starts a chain unless candidate i - 1 has the same diagonal, lies at most D query
// offsets before it and in the same bank sequence.  The threads of a warp (NW = 1) or of
// a block mark the chain heads in a bitmask (words at heads[], one per 32 candidates);
// each head's chain ends before the next head, and an HSP is emitted for every chain of
// length >= min_len.  Threads are tid, tid + nthreads, ...; sync() orders the two steps.
template <class Sync>
__device__ __forceinline__ void chain_emit(const uint64_t *cand, uint32_t nc, uint32_t *heads, uint32_t tid,
                                           uint32_t nthreads, Sync sync, uint32_t ql, uint32_t qa, int k, uint32_t D,
                                           uint32_t min_len, const SeqMap &sm, DevHsp *__restrict__ out,
                                           uint32_t *__restrict__ count, uint32_t out_cap,
                                           uint32_t *__restrict__ status) {
    const uint32_t nw = (nc + 31) / 32;
    for (uint32_t i0 = tid & ~31u; i0 < nw * 32; i0 += nthreads) {
        const uint32_t i = i0 + (tid & 31);
        bool head = false;
        if (i < nc) {
            const uint64_t key = cand[i];
            const uint32_t qs = (uint32_t)(key & 0xFFFFu);
            const uint64_t gpos = (key >> 16) - QBIAS + qs;
            head = true;
            if (i > 0) {
                const uint64_t prev = cand[i - 1];
                const uint32_t qp = (uint32_t)(prev & 0xFFFFu);
                if ((prev >> 16) == (key >> 16) && qs - qp <= D) {
                    const uint32_t sq = dev_seq_of(sm, gpos);
                    head = sm.start[sq] > gpos - (qs - qp);  // a sequence starts between them
                }
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, head);
        if ((tid & 31) == 0) heads[i0 / 32] = m;
    }
    sync();
    for (uint32_t i = tid; i < nc; i += nthreads) {
        if (!((heads[i / 32] >> (i & 31)) & 1u)) continue;
        // the next head after i
        uint32_t w = i / 32, rest = heads[w] & ~((2u << (i & 31)) - 1u);
        while (!rest && ++w < nw) rest = heads[w];
        const uint32_t end = (rest ? w * 32 + (uint32_t)(__ffs(rest) - 1) : nc) - 1;
        const uint64_t key = cand[i], kj = cand[end];
        const uint32_t qs = (uint32_t)(key & 0xFFFFu), qe = (uint32_t)(kj & 0xFFFFu) + (uint32_t)k;
        const uint32_t len = qe - qs;
        if (len < min_len) continue;
        const uint64_t gpos = (key >> 16) - QBIAS + qs;
        const uint32_t sq = dev_seq_of(sm, gpos);
        const uint32_t ds = (uint32_t)(gpos - sm.start[sq]);
        const uint32_t slot = atomicAdd(count, 1u);
        if (slot < out_cap) {
            DevHsp hh;
            hh.qi = qa + ql; hh.seq = sq; hh.qs = qs; hh.qe = qe; hh.ds = ds; hh.de = ds + len; hh.len = len;
            out[slot] = hh;
        } else {
            atomicOr(status, DEV_ERR_CAPACITY);
        }
    }
}
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// One warp per bucket.  Two bitmaps per warp mark diagonal hashes seen once and
// seen twice; hits whose hash was seen twice are candidates (a hash collision
// only adds a candidate that the exact chaining below then drops).  Candidates
// are sorted by (G', qpos) with a warp bitonic sort and chained.  Buckets with
// more than BGW_CAND candidates go to the global sort path.
constexpr int BGW_WARPS = 8;
constexpr int BGW_BITS = 8192;
constexpr int BGW_CAND = 256;
constexpr int BGC_CAND = 1024;  // entries a block-level bucket group takes

__global__ void __launch_bounds__(BGW_WARPS * 32) k_bucket_group_warp(
    const uint64_t *__restrict__ bkeys, const uint32_t *__restrict__ bcount, uint32_t bcap, uint32_t NB,
    const uint16_t *__restrict__ bq, uint32_t qa, int qbits, int k, uint32_t D, uint32_t min_len, int singles,
    SeqMap sm, DevHsp *__restrict__ out, uint32_t *__restrict__ count,
    uint32_t out_cap, uint64_t *__restrict__ ovf, unsigned long long ovf_cap,
    unsigned long long *__restrict__ ovf_count, uint32_t *__restrict__ status, uint32_t *__restrict__ next_bucket,
    uint32_t *__restrict__ big, uint32_t *__restrict__ big_count) {
    extern __shared__ __align__(16) unsigned char gw_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *seen = reinterpret_cast<uint32_t *>(gw_smem) + wib * (2 * BGW_BITS / 32);
    uint32_t *seen2 = seen + BGW_BITS / 32;
    uint64_t *cand = reinterpret_cast<uint64_t *>(gw_smem + BGW_WARPS * 2 * BGW_BITS / 8) + wib * BGW_CAND;
    uint32_t *heads = reinterpret_cast<uint32_t *>(gw_smem + BGW_WARPS * (2 * BGW_BITS / 8 + BGW_CAND * 8)) +
                      wib * (BGW_CAND / 32);
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(next_bucket, 1u);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= NB) break;
        const uint64_t beg = (uint64_t)b * bcap;
        const uint32_t total = bcount[b];
        const uint32_t n = min(total, bcap);
        if (total <= bcap && (n == 0 || (n == 1 && !singles))) continue;
        const uint32_t ql = bq[b];
        // a bucket that overflowed its capacity has entries in the spill list already: send the
        // stored part there as well, so that every (query, diagonal) stays on one path
        bool spill = total > bcap;
        uint32_t nc = 0;
        if (!singles && !spill) {
            for (int i = lane; i < BGW_BITS / 32; i += 32) { seen[i] = 0u; seen2[i] = 0u; }
            __syncwarp();
            for (uint32_t i0 = 0; i0 < n; i0 += 128) {
                uint64_t e[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t i = i0 + u * 32 + lane;
                    e[u] = i < n ? bkeys[beg + i] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (i0 + u * 32 + lane >= n) break;
                    const uint32_t h = (uint32_t)(((e[u] >> 16) * 0x9E3779B97F4A7C15ull) >> 51);  // 13 bits
                    const uint32_t bit = 1u << (h & 31);
                    const uint32_t old = atomicOr(&seen[h >> 5], bit);
                    if (old & bit) atomicOr(&seen2[h >> 5], bit);
                }
            }
            __syncwarp();
        }
        for (uint32_t i0 = 0; i0 < n && !spill; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint64_t key = 0;
            bool keep = false;
            if (i < n) {
                key = bkeys[beg + i];
                if (singles) {
                    keep = true;
                } else {
                    const uint32_t h = (uint32_t)(((key >> 16) * 0x9E3779B97F4A7C15ull) >> 51);  // 13 bits
                    keep = (seen2[h >> 5] >> (h & 31)) & 1u;
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, keep);
            if (nc + __popc(m) > BGW_CAND) {
                if (n <= BGC_CAND) {  // the block kernel takes it
                    if (lane == 0) big[atomicAdd(big_count, 1u)] = b;
                    nc = 0;
                    break;
                }
                spill = true;
            } else {
                if (keep) cand[nc + __popc(m & lt)] = key;
                nc += __popc(m);
            }
        }
        if (spill) {
            // too many candidates: hand the bucket to the global sort path, in its key format
            unsigned long long p0 = 0;
            if (lane == 0) p0 = atomicAdd(ovf_count, (unsigned long long)n);
            p0 = __shfl_sync(0xffffffffu, p0, 0);
            if (p0 + n <= ovf_cap) {  // else: counted only; the host enlarges the buffer and reruns
                for (uint32_t i = lane; i < n; i += 32) {
                    const uint64_t e = bkeys[beg + i];
                    ovf[p0 + i] = ((e >> 16) << (16 + qbits)) | ((uint64_t)ql << 16) | (e & 0xFFFFu);
                }
            }
            __syncwarp();
            continue;
        }
        if (nc < 2 && !singles) { __syncwarp(); continue; }
        if (nc == 0) { __syncwarp(); continue; }
        uint32_t P = 1;
        while (P < nc) P <<= 1;
        for (uint32_t i = nc + lane; i < P; i += 32) cand[i] = ~0ull;
        __syncwarp();
        for (uint32_t k2 = 2; k2 <= P; k2 <<= 1) {
            for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
                for (uint32_t i = lane; i < P; i += 32) {
                    const uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        const uint64_t a = cand[i], c = cand[ixj];
                        const bool up = (i & k2) == 0;
                        if ((a > c) == up) { cand[i] = c; cand[ixj] = a; }
                    }
                }
                __syncwarp();
            }
        }
        chain_emit(cand, nc, heads, lane, 32, WarpSync(), ql, qa, k, D, min_len, sm, out, count, out_cap, status);
        __syncwarp();
    }
}

// Exclusive prefix sum of v over the block (all threads call it); *total gets the sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_tot, uint32_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const uint32_t before = wid ? warp_tot[wid - 1] : 0u;
    __syncthreads();  // warp_tot is reused by the next call
    return before + x - v;
}

// One block per bucket that has more candidates than a warp holds (at most BGC_CAND
// entries in all): the same filter, sort and chaining as k_bucket_group_warp, over
// the whole block.  Blocks take the listed buckets in turn.
__global__ void __launch_bounds__(256) k_bucket_group_block(
    const uint64_t *__restrict__ bkeys, const uint32_t *__restrict__ bcount, uint32_t bcap,
    const uint16_t *__restrict__ bq, const uint32_t *__restrict__ big, const uint32_t *__restrict__ big_count,
    uint32_t qa, int k, uint32_t D, uint32_t min_len, int singles, SeqMap sm, DevHsp *__restrict__ out,
    uint32_t *__restrict__ count, uint32_t out_cap, uint32_t *__restrict__ status) {
    __shared__ uint32_t seen[BGW_BITS / 32], seen2[BGW_BITS / 32];
    __shared__ uint64_t cand[BGC_CAND];
    __shared__ uint32_t heads[BGC_CAND / 32];
    __shared__ uint32_t warp_tot[8];
    const uint32_t nbig = *big_count;
    for (uint32_t j = blockIdx.x; j < nbig; j += gridDim.x) {
        const uint32_t b = big[j];
        const uint64_t beg = (uint64_t)b * bcap;
        const uint32_t n = min(bcount[b], bcap);
        const uint32_t ql = bq[b];
        for (uint32_t i = threadIdx.x; i < BGW_BITS / 32; i += blockDim.x) { seen[i] = 0u; seen2[i] = 0u; }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t h = (uint32_t)(((bkeys[beg + i] >> 16) * 0x9E3779B97F4A7C15ull) >> 51);  // 13 bits
            const uint32_t bit = 1u << (h & 31);
            const uint32_t old = atomicOr(&seen[h >> 5], bit);
            if (old & bit) atomicOr(&seen2[h >> 5], bit);
        }
        __syncthreads();
        uint32_t nc = 0;
        for (uint32_t i0 = 0; i0 < n; i0 += blockDim.x) {
            const uint32_t i = i0 + threadIdx.x;
            uint64_t key = 0;
            bool keep = false;
            if (i < n) {
                key = bkeys[beg + i];
                const uint32_t h = (uint32_t)(((key >> 16) * 0x9E3779B97F4A7C15ull) >> 51);
                keep = singles || ((seen2[h >> 5] >> (h & 31)) & 1u);
            }
            uint32_t tot = 0;
            const uint32_t pos = nc + block_excl_scan(keep ? 1u : 0u, warp_tot, tot);
            if (keep) cand[pos] = key;
            nc += tot;
        }
        uint32_t P = 1;
        while (P < nc) P <<= 1;
        for (uint32_t i = nc + threadIdx.x; i < P; i += blockDim.x) cand[i] = ~0ull;
        __syncthreads();
        for (uint32_t k2 = 2; k2 <= P; k2 <<= 1) {
            for (uint32_t jj = k2 >> 1; jj > 0; jj >>= 1) {
                for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                    const uint32_t ixj = i ^ jj;
                    if (ixj > i) {
                        const uint64_t x = cand[i], y = cand[ixj];
                        if ((x > y) == ((i & k2) == 0)) { cand[i] = y; cand[ixj] = x; }
                    }
                }
                __syncthreads();
            }
        }
        chain_emit(cand, nc, heads, threadIdx.x, blockDim.x, BlockSync(), ql, qa, k, D, min_len, sm, out, count,
                   out_cap, status);
        __syncthreads();
    }
}

// quadruples (query, qpos, seq, pos) of sorted hits (tests)
__global__ void k_decode_hits(const uint64_t *__restrict__ keys, uint64_t n, int qbits, uint32_t qa,
                              const uint64_t *__restrict__ seq_start, uint32_t n_seqs, uint32_t *__restrict__ out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    HitKey h = dec_key(keys[i], qbits);
    uint64_t gpos = h.gkey - QBIAS + h.qpos;
    uint32_t sq = dev_upper_index(seq_start, n_seqs + 1, gpos);
    out[4 * i + 0] = qa + h.ql;
    out[4 * i + 1] = h.qpos;
    out[4 * i + 2] = sq;
    out[4 * i + 3] = (uint32_t)(gpos - seq_start[sq]);
}

// --------------------------------------------------- a9: X-drop extension --
__device__ __forceinline__ int32_t dev_pair(uint32_t a, uint32_t b, int32_t match, int32_t mismatch) {
    return (a < 4u && a == b) ? match : mismatch;
}

// Walks packed bases one at a time, reloading the code word every 16 bases and the
// non-base word every 32 (instead of two loads per base).
struct BaseCursor {
    const uint32_t *pk, *nb;
    uint64_t wpk_i = ~0ull, wnb_i = ~0ull;
    uint32_t wpk = 0, wnb = 0;
    __device__ __forceinline__ BaseCursor(const uint32_t *p, const uint32_t *n) : pk(p), nb(n) {}
    __device__ __forceinline__ uint32_t at(uint64_t g) {  // 2-bit code, or 4 for a non-base
        const uint64_t a = g >> 4, b = g >> 5;
        if (a != wpk_i) { wpk_i = a; wpk = pk[a]; }
        if (b != wnb_i) { wnb_i = b; wnb = nb[b]; }
        return ((wnb >> (g & 31)) & 1u) ? 4u : (wpk >> (30 - 2 * (int)(g & 15))) & 3u;
    }
};

// One direction of the X-drop walk, 32 steps per round for a whole warp.  Step e
// (1-based) compares query base qg(e) with bank base dg(e).  The sequential rule
// (score += s; if score > best: best = score, ext = e; else if best - score > X:
// stop) stops at the first e where max(best so far, score_e) - score_e > X, and
// ext is the first step that reached the final best.  Returns ext.
// The walk continues a lane's walk: steps e_first.. with the score, best and ext that the
// steps before e_first left (0, 0, 0 and e_first = 1 for a fresh walk).
template <int DIR>
__device__ __forceinline__ uint32_t xdrop_walk_warp(const uint32_t *__restrict__ qpk, const uint32_t *__restrict__ qnb,
                                                    const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                                    uint64_t qg0, uint64_t dg0, uint32_t emax, int32_t match,
                                                    int32_t mismatch, int32_t X, int lane, uint32_t e_first,
                                                    int32_t score0, int32_t best0, uint32_t ext0) {
    int32_t carry_score = score0, carry_best = best0;
    uint32_t carry_ext = ext0;
    for (uint32_t e0 = e_first; e0 <= emax; e0 += 32) {
        const uint32_t e = e0 + lane;
        const bool in = e <= emax;
        int32_t sc = 0;
        if (in) {
            const uint64_t qg = DIR > 0 ? qg0 + (e - 1) : qg0 - e;
            const uint64_t dg = DIR > 0 ? dg0 + (e - 1) : dg0 - e;
            sc = dev_pair(dev_base(qpk, qnb, qg), dev_base(bpk, bnb, dg), match, mismatch);
        }
        // running score (inclusive prefix sum) and running best (inclusive prefix max)
        int32_t S = sc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, S, o);
            if (lane >= o) S += t;
        }
        S += carry_score;
        int32_t M = in ? S : INT32_MIN;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, M, o);
            if (lane >= o) M = max(M, t);
        }
        M = max(M, carry_best);
        const uint32_t stop = __ballot_sync(0xffffffffu, in && M - S > X);
        const uint32_t last = stop ? (uint32_t)(__ffs(stop) - 1) : 31u;  // last lane that counts this round
        const int32_t Mlast = __shfl_sync(0xffffffffu, M, last);
        if (Mlast > carry_best) {
            // first step of this round that reached the new best
            const uint32_t hit = __ballot_sync(0xffffffffu, in && (uint32_t)lane <= last && S == Mlast);
            carry_ext = e0 + (uint32_t)(__ffs(hit) - 1);
            carry_best = Mlast;
        }
        if (stop) break;
        carry_score = __shfl_sync(0xffffffffu, S, 31);
    }
    return carry_ext;
}

// 16 bases from position p (p >= -16; bases before 0 read as code 0, non-base): 2-bit
// codes with base p in bits 31-30, and a mask with bit i set when base p + i is a non-base.
// The packed arrays carry two words past the last base, so p + 15 may pass the end.
__device__ __forceinline__ void base_window16(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb,
                                             int64_t p, uint32_t &codes, uint32_t &bad) {
    const int64_t a = p >> 4, b = p >> 5;  // floor division
    const uint32_t w0 = a >= 0 ? pk[a] : 0u, w1 = pk[a + 1];
    const uint32_t off = (uint32_t)(p & 15);
    codes = (uint32_t)((((uint64_t)w0 << 32) | w1) >> (32 - 2 * off));
    const uint32_t n0 = b >= 0 ? nb[b] : 0xFFFFFFFFu, n1 = nb[b + 1];
    bad = (uint32_t)(((((uint64_t)n1) << 32) | n0) >> (uint32_t)(p & 31)) & 0xFFFFu;
}

// One direction of the walk on one lane, by the sequential rule, for at most lim steps,
// 16 steps per window of bases: returns whether the walk ended (the drop passed X, or the
// sequence ended); score, best, ext and the steps taken are left for a continuation.
template <int DIR>
__device__ __forceinline__ bool xdrop_walk_lane(const uint32_t *__restrict__ qpk, const uint32_t *__restrict__ qnb,
                                                const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                                uint64_t qg0, uint64_t dg0, uint32_t emax, int32_t match,
                                                int32_t mismatch, int32_t X, uint32_t lim, int32_t &score,
                                                int32_t &best, uint32_t &ext, uint32_t &steps) {
    score = 0;
    best = 0;
    ext = 0;
    const uint32_t until = min(emax, lim);
    for (uint32_t e0 = 0; e0 < until; e0 += 16) {
        // steps e0 + 1 .. e0 + 16: positions qg0 + e0 .. + 15 (right), qg0 - e0 - 16 .. - 1 (left)
        const int64_t qp = DIR > 0 ? (int64_t)(qg0 + e0) : (int64_t)qg0 - (int64_t)e0 - 16;
        const int64_t dp = DIR > 0 ? (int64_t)(dg0 + e0) : (int64_t)dg0 - (int64_t)e0 - 16;
        uint32_t wq, bq, wd, bd;
        base_window16(qpk, qnb, qp, wq, bq);
        base_window16(bpk, bnb, dp, wd, bd);
        const uint32_t x = ~(wq ^ wd), eq = x & (x >> 1);  // bit 30 - 2k: codes equal at window base k
        const uint32_t bad = bq | bd;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const uint32_t e = e0 + (uint32_t)t + 1;
            if (e > until) {
                steps = until;
                return until == emax;
            }
            const int k = DIR > 0 ? t : 15 - t;
            const bool same = ((eq >> (30 - 2 * k)) & 1u) && !((bad >> k) & 1u);
            score += same ? match : mismatch;
            if (score > best) {
                best = score;
                ext = e;
            } else if (best - score > X) {
                steps = e;
                return true;
            }
        }
    }
    steps = until;
    return until == emax;
}

// X-drop extension of both ends of every HSP.  Each lane walks one HSP's ends on its own
// (most walks end within a few dozen steps) for at most lim steps each; the warp then
// continues the walks that did not end, one after the other, 32 steps per round.
__global__ void k_xdrop(DevHsp *__restrict__ h, uint32_t n, const uint32_t *__restrict__ qpk,
                        const uint32_t *__restrict__ qnb, const uint64_t *__restrict__ qstart,
                        const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                        const uint64_t *__restrict__ seq_start, int32_t match, int32_t mismatch, int32_t X,
                        uint32_t nq, uint32_t n_seqs, uint32_t lim, uint32_t *__restrict__ next_group) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        // groups of 32 HSPs from a counter: a warp whose group held long walks takes fewer
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(next_group, 1u);
        const uint32_t b0 = __shfl_sync(0xffffffffu, g, 0) * 32u;
        if (b0 >= n) break;
        const uint32_t i = b0 + lane;
        bool valid = i < n;
        DevHsp r;
        uint64_t qb = 0, sb = 0;
        uint32_t emax_l = 0, emax_r = 0;
        if (valid) {
            r = h[i];
            valid = GN_CHECK(r.qi < nq && r.seq < n_seqs);
        }
        if (valid) {
            qb = qstart[r.qi];
            sb = seq_start[r.seq];
            const uint32_t m = (uint32_t)(qstart[r.qi + 1] - qb), L = (uint32_t)(seq_start[r.seq + 1] - sb);
            emax_l = min(r.qs, r.ds);
            emax_r = min(m - r.qe, L - r.de);
        }
        int32_t sl = 0, bl = 0, sr = 0, br = 0;
        uint32_t el = 0, er = 0, nl = 0, nr = 0;
        bool done_l = true, done_r = true;
        if (valid) {
            done_l = xdrop_walk_lane<-1>(qpk, qnb, bpk, bnb, qb + r.qs, sb + r.ds, emax_l, match, mismatch, X, lim, sl,
                                         bl, el, nl);
            done_r = xdrop_walk_lane<1>(qpk, qnb, bpk, bnb, qb + r.qe, sb + r.de, emax_r, match, mismatch, X, lim, sr,
                                        br, er, nr);
        }
        // walks that did not end: the whole warp continues them
        uint32_t todo = __ballot_sync(0xffffffffu, !done_l || !done_r);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint64_t q0 = __shfl_sync(0xffffffffu, qb, src), s0 = __shfl_sync(0xffffffffu, sb, src);
            const bool cl = __shfl_sync(0xffffffffu, !done_l, src), cr = __shfl_sync(0xffffffffu, !done_r, src);
            if (cl) {
                const uint32_t qs = __shfl_sync(0xffffffffu, valid ? r.qs : 0u, src);
                const uint32_t ds = __shfl_sync(0xffffffffu, valid ? r.ds : 0u, src);
                const uint32_t x = xdrop_walk_warp<-1>(
                    qpk, qnb, bpk, bnb, q0 + qs, s0 + ds, __shfl_sync(0xffffffffu, emax_l, src), match, mismatch, X,
                    lane, __shfl_sync(0xffffffffu, nl, src) + 1, __shfl_sync(0xffffffffu, sl, src),
                    __shfl_sync(0xffffffffu, bl, src), __shfl_sync(0xffffffffu, el, src));
                if (lane == src) el = x;
            }
            if (cr) {
                const uint32_t qe = __shfl_sync(0xffffffffu, valid ? r.qe : 0u, src);
                const uint32_t de = __shfl_sync(0xffffffffu, valid ? r.de : 0u, src);
                const uint32_t x = xdrop_walk_warp<1>(
                    qpk, qnb, bpk, bnb, q0 + qe, s0 + de, __shfl_sync(0xffffffffu, emax_r, src), match, mismatch, X,
                    lane, __shfl_sync(0xffffffffu, nr, src) + 1, __shfl_sync(0xffffffffu, sr, src),
                    __shfl_sync(0xffffffffu, br, src), __shfl_sync(0xffffffffu, er, src));
                if (lane == src) er = x;
            }
        }
        if (valid) {
            r.qs -= el; r.ds -= el;
            r.qe += er; r.de += er;
            r.len = min(r.qe - r.qs, r.de - r.ds);
            h[i] = r;
        }
    }
}

// ------------------------------------------- long queries: segments, join --
// Bases of each segment (block v): len bytes from offset off[v] of query parent[v].
__global__ void k_segment_bases(const uint8_t *__restrict__ qbases, const uint64_t *__restrict__ qstart,
                                const uint32_t *__restrict__ parent, const uint64_t *__restrict__ off,
                                const uint64_t *__restrict__ vstart, uint8_t *__restrict__ out) {
    const uint32_t v = blockIdx.x;
    const uint64_t from = qstart[parent[v]] + off[v], to = vstart[v], len = vstart[v + 1] - to;
    for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) out[to + i] = qbases[from + i];
}

// Chain pieces of the segments onto their queries; the len word carries the diagonal
// (ds - qs mod 2^32, distinct for distinct diagonals when sequences are shorter than
// 2^32 - 2^24 bases) for the join's sort.
__global__ void k_segment_map(DevHsp *__restrict__ h, uint32_t n, const uint32_t *__restrict__ parent,
                              const uint64_t *__restrict__ off) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DevHsp r = h[i];
    const uint32_t o = (uint32_t)off[r.qi];
    r.qi = parent[r.qi];
    r.qs += o;
    r.qe += o;
    r.len = r.ds - r.qs;
    h[i] = r;
}

// Pieces sorted by (qi, seq, diagonal, qs).  Two pieces of one chain share a hit, so
// a piece joins the current chain when its first hit starts no later than the chain's
// last hit (qs + span <= qe); pieces of different chains on one diagonal are more than
// D >= 0 offsets apart and never do.  The first piece of each (qi, seq, diagonal) run
// walks the run.  A chain is written at the index of its first piece and kept (flag)
// when it is at least min_len long.
__global__ void k_stitch_sweep(const DevHsp *__restrict__ in, uint32_t n, uint32_t span, uint32_t min_len,
                               DevHsp *__restrict__ out, uint32_t *__restrict__ flag) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    auto same = [&](uint32_t a, uint32_t b) {
        return in[a].qi == in[b].qi && in[a].seq == in[b].seq && in[a].len == in[b].len;
    };
    if (i > 0 && same(i - 1, i)) return;
    uint32_t j = i;
    while (j < n && same(j, i)) {
        DevHsp c = in[j];
        const uint32_t head = j++;
        while (j < n && same(j, i) && in[j].qs + span <= c.qe) {
            c.qe = max(c.qe, in[j].qe);
            flag[j++] = 0;
        }
        c.len = c.qe - c.qs;
        c.de = c.ds + c.len;
        out[head] = c;
        flag[head] = c.len >= min_len ? 1u : 0u;
    }
}

// -------------------------------------------------- a10: overlap merging --
// Records sorted by (qi, seq, qs).  The first record of each (qi, seq) run sweeps
// the run in (qs, ds, qe) order (records of one qs, rarely more than one, are taken
// by increasing (ds, qe); de = ds + qe - qs for these ungapped HSPs, so records
// equal in (ds, qe) are equal): each record joins the current box when both its
// query and bank ranges intersect the box, otherwise it starts a new box.  The
// run's boxes are written, in that order, at its first indices, flagged 1; its
// other indices are flagged 0.
__device__ __forceinline__ uint64_t ov_key(const DevHsp &h) { return ((uint64_t)h.ds << 32) | h.qe; }

__global__ void k_overlap_sweep(const DevHsp *__restrict__ in, uint32_t n, DevHsp *__restrict__ out,
                                uint32_t *__restrict__ flag) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t qi = in[i].qi, seq = in[i].seq;
    if (i > 0 && in[i - 1].qi == qi && in[i - 1].seq == seq) return;  // not the head of a run
    uint32_t o = i;  // next box slot
    bool open = false;
    DevHsp box{};  // set by the run's first record
    auto visit = [&](const DevHsp &h) {
        if (open && h.qs < box.qe && box.qs < h.qe && h.ds < box.de && box.ds < h.de) {
            box.qs = min(box.qs, h.qs);
            box.qe = max(box.qe, h.qe);
            box.ds = min(box.ds, h.ds);
            box.de = max(box.de, h.de);
            return;
        }
        if (open) {
            box.len = min(box.qe - box.qs, box.de - box.ds);
            out[o] = box;
            flag[o++] = 1;
        }
        box = h;
        open = true;
    };
    uint32_t g0 = i;
    while (g0 < n && in[g0].qi == qi && in[g0].seq == seq) {
        const uint32_t qs = in[g0].qs;
        uint32_t g1 = g0 + 1;
        while (g1 < n && in[g1].qi == qi && in[g1].seq == seq && in[g1].qs == qs) ++g1;
        if (g1 - g0 == 1) {
            visit(in[g0]);
        } else {
            // the group's records by increasing (ds, qe), then index: each step takes the
            // smallest (key, index) above the last one taken
            uint64_t last_k = 0;
            uint32_t last_j = 0;
            for (uint32_t t = g0; t < g1; ++t) {
                uint64_t best_k = ~0ull;
                uint32_t best_j = g1;
                for (uint32_t j = g0; j < g1; ++j) {
                    const uint64_t kj = ov_key(in[j]);
                    const bool after = t == g0 || kj > last_k || (kj == last_k && j > last_j);
                    if (after && (kj < best_k || (kj == best_k && j < best_j))) {
                        best_k = kj;
                        best_j = j;
                    }
                }
                visit(in[best_j]);
                last_k = best_k;
                last_j = best_j;
            }
        }
        g0 = g1;
    }
    box.len = min(box.qe - box.qs, box.de - box.ds);
    out[o] = box;
    flag[o++] = 1;
    for (uint32_t j = o; j < g0; ++j) flag[j] = 0;
}

// ----------------------------------------------------- a11: selection --
// Per-query selection on records sorted by (qi, seq, qs, ds, qe, de): a block per
// query keeps its N longest records, ties broken by that order (a stable choice by
// length), and writes them by (length desc, seq, qs, ds, qe, de).  The N-th largest
// length T comes from two 256-bin histograms (high and low byte of the length); the
// selected records are those longer than T and the first ones of length T.
constexpr int SQ_CAP = 1024;  // largest N this kernel handles
constexpr int SQ_THREADS = 512;

__global__ void __launch_bounds__(SQ_THREADS) k_select_query(const DevHsp *__restrict__ rec,
                                                             const uint32_t *__restrict__ qfirst,
                                                             const uint64_t *__restrict__ qout, uint32_t N,
                                                             DevHsp *__restrict__ sel) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t warp_tot[SQ_THREADS / 32];
    __shared__ uint64_t keys[SQ_CAP];
    __shared__ uint32_t T_s, gt_s;
    const uint32_t q = blockIdx.x;
    const uint32_t a = qfirst[q], b = qfirst[q + 1], n = b - a;
    const uint64_t out0 = qout[q];
    const uint32_t nsel = (uint32_t)(qout[q + 1] - out0);
    if (nsel == 0) return;
    uint32_t T = 0, r_eq = n;  // n <= N: every record is selected
    if (n > N) {
        uint32_t above = 0, hb = 0;
        for (int level = 0; level < 2; ++level) {
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            // one shared-memory atomic per distinct bin of a warp's 32 records (lengths are
            // concentrated in few bins)
            for (uint32_t i0 = a + (threadIdx.x & ~31u); i0 < b; i0 += blockDim.x) {
                const uint32_t i = i0 + (threadIdx.x & 31u);
                uint32_t bin = 256u;
                if (i < b) {
                    const uint32_t len = min(rec[i].len, 65535u);
                    if (level == 0) bin = len >> 8;
                    else if ((len >> 8) == hb) bin = len & 0xFFu;
                }
                const uint32_t peers = __match_any_sync(0xffffffffu, bin);
                if (bin < 256u && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
                    atomicAdd(&hist[bin], (uint32_t)__popc(peers));
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t acc = above;
                int x = 255;
                while (acc + hist[x] < N) acc += hist[x--];
                T_s = level == 0 ? (uint32_t)x : ((hb << 8) | (uint32_t)x);
                gt_s = acc;
            }
            __syncthreads();
            if (level == 0) { hb = T_s; above = gt_s; }
            else { T = T_s; above = gt_s; }
            __syncthreads();
        }
        r_eq = N - above;  // records of length T to take, in array order
    }
    // ordered compaction of the selected records (array order), keyed by (length desc, position):
    // each thread takes a contiguous run of records, counts its records longer than T and of
    // length T, and two block scans give its first output slot and its first rank among the
    // records of length T
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    uint32_t n_gt = 0, n_eq = 0;
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t len = min(rec[a + i].len, 65535u);
        const bool gt = n <= N || len > T;
        n_gt += gt ? 1u : 0u;
        n_eq += (!gt && len == T) ? 1u : 0u;
    }
    uint32_t tot = 0;
    uint32_t eq_rank = block_excl_scan(n_eq, warp_tot, tot);
    const uint32_t n_take = n_gt + min(n_eq, r_eq > eq_rank ? r_eq - eq_rank : 0u);
    uint32_t pos = block_excl_scan(n_take, warp_tot, tot);
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t len = min(rec[a + i].len, 65535u);
        const bool gt = n <= N || len > T;
        const bool eq = !gt && len == T;
        const bool take = gt || (eq && eq_rank < r_eq);
        eq_rank += eq ? 1u : 0u;
        if (take) keys[pos++] = ((uint64_t)(65535u - len) << 32) | i;
    }
    __syncthreads();
    // bitonic sort of the nsel keys (unique: they carry the position)
    uint32_t P = 1;
    while (P < nsel) P <<= 1;
    for (uint32_t i = nsel + threadIdx.x; i < P; i += blockDim.x) keys[i] = ~0ull;
    __syncthreads();
    for (uint32_t k2 = 2; k2 <= P; k2 <<= 1) {
        for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = keys[i], y = keys[ixj];
                    if ((x > y) == ((i & k2) == 0)) { keys[i] = y; keys[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t k = threadIdx.x; k < nsel; k += blockDim.x) sel[out0 + k] = rec[a + (uint32_t)(keys[k] & 0xFFFFFFFFu)];
}

// first[q] = first record of query q in records sorted by query (first[nq] = n), and, when
// cnt is given, cnt[q] = min(N, records of query q): the counts of the selected records
__device__ __forceinline__ uint32_t first_of_query(const DevHsp *__restrict__ rec, uint32_t n, uint32_t q) {
    uint32_t lo = 0, hi = n;  // first index with qi >= q
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (rec[mid].qi < q) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_query_bounds(const DevHsp *__restrict__ rec, uint32_t n, uint32_t nq, uint32_t *__restrict__ first,
                               uint32_t N, uint32_t *__restrict__ cnt) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > nq) return;
    const uint32_t f = first_of_query(rec, n, q);
    first[q] = f;
    if (cnt && q < nq) cnt[q] = min(N, first_of_query(rec, n, q + 1) - f);
}

__global__ void k_first_of_query(const uint32_t *__restrict__ recs, int W, uint32_t n, uint32_t *__restrict__ first) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q = recs[(uint64_t)i * W];
    if (i == 0 || recs[(uint64_t)(i - 1) * W] != q) first[q] = i;
}

__global__ void k_select_flags(const DevHsp *__restrict__ h, uint32_t n, const uint32_t *__restrict__ first,
                               uint32_t N, uint32_t *__restrict__ flag) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (N == 0 || i - first[h[i].qi] < N) ? 1u : 0u;
}

// -------------------------------------------- a12: banded Smith-Waterman --
// One warp per selected HSP.  Lanes own band offsets b (diagonal j - i = dlo + b);
// rows i of the DP window are processed in order, each row in chunks of 32
// offsets.  The previous row (H, E and their start cells) lives in a per-HSP
// scratch strip of B entries.  Horizontal gaps (F) inside a row are resolved
// by a warp max-scan of X(b') = H0(b') + go + ge - ge*b' (H0 = the cell's best
// over 0, diagonal and vertical gap), since F(b) = max_{b'<b} X(b') + ge*(b-1)
// reproduces the sequential recurrence, including its "open wins ties" choice
// when the scan keeps the later of equal values.
struct SwCell {
    int32_t H, E;
    uint32_t SH, SE;  // start cells: (row - I0) * B + band offset
};

constexpr int32_t SW_NEG = -(1 << 29);
constexpr int32_t SW_XNEG = -(1 << 30);

__device__ __forceinline__ void scan_pair_max(int32_t &v, uint32_t &s, int lane) {
    // inclusive scan, later lane wins ties
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t ov = __shfl_up_sync(0xffffffffu, v, o);
        uint32_t os = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o && ov > v) { v = ov; s = os; }
    }
}


// Band of at most 64 diagonals: lane l owns the two adjacent band offsets 2l and
// 2l+1 and keeps their previous-row states in registers.  The vertical-gap input of
// offset 2l is the lane's own offset 2l+1; that of 2l+1 comes from the next lane.
// One warp max-scan per row resolves horizontal gaps for all 64 offsets: each lane
// contributes the later-wins maximum of its two X values.  Bases are read through
// per-lane word cursors (one load per 16 rows).
__device__ __forceinline__ void sw_rows_pair(int64_t I0, int64_t I1, int64_t J0, int64_t J1, int64_t dlo, int64_t B,
                                             uint64_t qb, uint64_t sb, const uint32_t *__restrict__ qpk,
                                             const uint32_t *__restrict__ qnb, const uint32_t *__restrict__ bpk,
                                             const uint32_t *__restrict__ bnb, int32_t match, int32_t mismatch,
                                             int32_t goe, int32_t ge, int lane, int32_t &best, int64_t &bi,
                                             int64_t &bj, uint32_t &bs) {
    int32_t pH0 = 0, pE0 = SW_NEG, pH1 = 0, pE1 = SW_NEG;
    uint32_t pSH0 = 0, pSE0 = 0, pSH1 = 0, pSE1 = 0;
    const int32_t b0 = 2 * lane, b1 = 2 * lane + 1;
    BaseCursor cq(qpk, qnb), cd(bpk, bnb);
    const int32_t irows = (int32_t)(I1 - I0);
    const uint32_t Bu = (uint32_t)B;  // start cells: row * B + band offset
    const int32_t jlo = (int32_t)(J0 - I0 - dlo), jhi = (int32_t)(J1 - 1 - I0 - dlo);  // band offset limits at row I0
    for (int32_t r = 0; r < irows; ++r) {
        // row i = I0 + r: band offsets with J0 <= i + dlo + b <= J1 - 1
        const int32_t blo = max(0, jlo - r), bhi = min((int32_t)B - 1, jhi - r);
        if (blo > bhi) continue;
        const bool prow = r > 0;
        const int32_t pblo = max(0, jlo - r + 1), pbhi = min((int32_t)B - 1, jhi - r + 1);
        const uint64_t i = (uint64_t)(I0 + r);
        const uint32_t qc = cq.at(qb + i);
        // previous-row state at offset b1 + 1 = next lane's b0
        const int32_t uH = __shfl_down_sync(0xffffffffu, pH0, 1), uE = __shfl_down_sync(0xffffffffu, pE0, 1);
        const uint32_t uSH = __shfl_down_sync(0xffffffffu, pSH0, 1), uSE = __shfl_down_sync(0xffffffffu, pSE0, 1);
        const bool act0 = b0 >= blo && b0 <= bhi, act1 = b1 >= blo && b1 <= bhi;
        const uint64_t j0g = sb + (uint64_t)((int64_t)i + dlo + b0);
        uint32_t d0 = 4u, d1 = 4u;
        if (act0) d0 = cd.at(j0g);
        if (act1) d1 = cd.at(j0g + 1);
        // cell b0
        int32_t E0 = SW_NEG;
        uint32_t SE0 = 0;
        if (act0 && prow && b1 >= pblo && b1 <= pbhi) {
            const int32_t eo = pH1 + goe, ee = pE1 + ge;
            if (eo >= ee) { E0 = eo; SE0 = pSH1; } else { E0 = ee; SE0 = pSE1; }
        }
        const bool okd0 = act0 && prow && b0 >= pblo && b0 <= pbhi;
        const int32_t Hd0 = okd0 ? pH0 : 0;
        const uint32_t SD0 = (Hd0 > 0) ? pSH0 : (uint32_t)r * Bu + (uint32_t)b0;
        const int32_t Dg0 = Hd0 + dev_pair(qc, d0, match, mismatch);
        int32_t c0v; uint32_t c0s;
        if (Dg0 >= E0) { c0v = Dg0; c0s = SD0; } else { c0v = E0; c0s = SE0; }
        const int32_t H00 = c0v > 0 ? c0v : 0;
        // cell b1
        int32_t E1 = SW_NEG;
        uint32_t SE1 = 0;
        if (act1 && prow && b1 + 1 >= pblo && b1 + 1 <= pbhi) {
            const int32_t eo = uH + goe, ee = uE + ge;
            if (eo >= ee) { E1 = eo; SE1 = uSH; } else { E1 = ee; SE1 = uSE; }
        }
        const bool okd1 = act1 && prow && b1 >= pblo && b1 <= pbhi;
        const int32_t Hd1 = okd1 ? pH1 : 0;
        const uint32_t SD1 = (Hd1 > 0) ? pSH1 : (uint32_t)r * Bu + (uint32_t)b1;
        const int32_t Dg1 = Hd1 + dev_pair(qc, d1, match, mismatch);
        int32_t c1v; uint32_t c1s;
        if (Dg1 >= E1) { c1v = Dg1; c1s = SD1; } else { c1v = E1; c1s = SE1; }
        const int32_t H01 = c1v > 0 ? c1v : 0;
        // horizontal gaps: F(b) = max_{b'<b} X(b') + ge*(b-1), X(b') = H0(b') + go + ge - ge*b'
        const int32_t x0 = act0 ? H00 + goe - ge * b0 : SW_XNEG;
        const int32_t x1 = act1 ? H01 + goe - ge * b1 : SW_XNEG;
        int32_t xv = x1 >= x0 ? x1 : x0;
        uint32_t xs = x1 >= x0 ? c1s : c0s;
        scan_pair_max(xv, xs, lane);
        int32_t ev = __shfl_up_sync(0xffffffffu, xv, 1);
        uint32_t es = __shfl_up_sync(0xffffffffu, xs, 1);
        if (lane == 0) { ev = SW_XNEG; es = 0; }
        const int32_t F0 = (ev > SW_XNEG) ? ev + ge * (b0 - 1) : SW_NEG;
        const uint32_t SF0 = es;
        int32_t e1v = ev;
        uint32_t e1s = es;
        if (x0 >= e1v) { e1v = x0; e1s = c0s; }
        const int32_t F1 = (e1v > SW_XNEG) ? e1v + ge * (b1 - 1) : SW_NEG;
        int32_t H0v, H1v;
        uint32_t S0, S1;
        if (H00 >= F0) { H0v = H00; S0 = c0s; } else { H0v = F0; S0 = SF0; }
        if (H01 >= F1) { H1v = H01; S1 = c1s; } else { H1v = F1; S1 = e1s; }
        if (act0 && H0v > best) { best = H0v; bi = (int64_t)i; bj = (int64_t)i + dlo + b0; bs = S0; }
        if (act1 && H1v > best) { best = H1v; bi = (int64_t)i; bj = (int64_t)i + dlo + b1; bs = S1; }
        pH0 = H0v; pE0 = E0; pSH0 = S0; pSE0 = SE0;
        pH1 = H1v; pE1 = E1; pSH1 = S1; pSE1 = SE1;
    }
}


// Band width (diagonals) of an HSP's alignment: the spread of its end diagonals plus 2w + 1.
__device__ __forceinline__ int64_t dev_band(const DevHsp &h, int32_t w) {
    const int64_t d_s = (int64_t)h.ds - h.qs, d_e = (int64_t)h.de - h.qe;
    return max(d_s, d_e) - min(d_s, d_e) + 2 * (int64_t)w + 1;
}

// One HSP aligned by a whole warp: the pair path (bands of at most 64 diagonals), or
// with STRIP the strip path (the band in chunks of 32 offsets, previous row in scratch).
template <bool STRIP>
__device__ void sw_task_warp(const DevHsp *__restrict__ sel, uint32_t task, const uint64_t *__restrict__ strip_off,
                             SwCell *__restrict__ strips, const uint32_t *__restrict__ qpk,
                             const uint32_t *__restrict__ qnb, const uint64_t *__restrict__ qstart,
                             const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                             const uint64_t *__restrict__ seq_start, int32_t match, int32_t mismatch, int32_t go,
                             int32_t ge, int32_t w, DevAln *__restrict__ out, uint32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const DevHsp h = sel[task];
    const uint64_t qb = qstart[h.qi], sb = seq_start[h.seq];
    const int64_t m = (int64_t)(qstart[h.qi + 1] - qb), L = (int64_t)(seq_start[h.seq + 1] - sb);
    const int64_t d_s = (int64_t)h.ds - h.qs, d_e = (int64_t)h.de - h.qe;
    const int64_t dlo = min(d_s, d_e) - w, dhi = max(d_s, d_e) + w;
    const int64_t I0 = max((int64_t)0, (int64_t)h.qs - w), I1 = min(m, (int64_t)h.qe + w);
    const int64_t J0 = max((int64_t)0, (int64_t)h.ds - w), J1 = min(L, (int64_t)h.de + w);
    const int64_t B = dhi - dlo + 1;
    DevAln res;
    res.qi = h.qi; res.seq = h.seq; res.qs = res.qe = res.ds = res.de = 0; res.score = 0; res.pad = 0;
    // start cells are (row - I0) * B + offset in 32 bits; strips hold up to 65,536 entries
    if (B > 65535 || (uint64_t)max(I1 - I0, (int64_t)0) * (uint64_t)B >= (1ull << 32)) {
        if (lane == 0) { atomicOr(status, DEV_ERR_BAND_TOO_WIDE); out[task] = res; }
        return;
    }
    SwCell *row = strips + strip_off[task];
    int32_t best = 0;
    int64_t bi = INT64_MAX, bj = INT64_MAX;
    uint32_t bs = 0;
    const int32_t goe = go + ge;
    if (!STRIP) {  // bands of at most 64 diagonals (the caller routes wider ones elsewhere)
        sw_rows_pair(I0, I1, J0, J1, dlo, B, qb, sb, qpk, qnb, bpk, bnb, match, mismatch, goe, ge, lane, best, bi,
                     bj, bs);
    } else
    for (int64_t i = I0; i < I1; ++i) {
        const int64_t blo = max((int64_t)0, J0 - i - dlo), bhi = min(B - 1, J1 - 1 - i - dlo);
        if (blo > bhi) continue;
        const bool prow = i - 1 >= I0;
        const int64_t pblo = max((int64_t)0, J0 - (i - 1) - dlo), pbhi = min(B - 1, J1 - 1 - (i - 1) - dlo);
        const uint32_t qc = dev_base(qpk, qnb, qb + (uint64_t)i);
        int32_t carry_v = SW_XNEG;
        uint32_t carry_s = 0;
        for (int64_t c0 = blo; c0 <= bhi; c0 += 32) {
            const int64_t b = c0 + lane;
            const bool act = b <= bhi;
            SwCell pd{0, SW_NEG, 0, 0}, pu{0, SW_NEG, 0, 0};
            const bool ok_d = act && prow && b >= pblo && b <= pbhi;
            const bool ok_u = act && prow && b + 1 >= pblo && b + 1 <= pbhi;
            if (ok_d) pd = row[b];
            if (ok_u) pu = row[b + 1];
            __syncwarp();
            int32_t E = SW_NEG;
            uint32_t SE = 0;
            if (ok_u) {
                int32_t eo = pu.H + goe, ee = pu.E + ge;
                if (eo >= ee) { E = eo; SE = pu.SH; } else { E = ee; SE = pu.SE; }
            }
            const int32_t Hd = ok_d ? pd.H : 0;
            const uint32_t SD = (Hd > 0) ? pd.SH : (uint32_t)(i - I0) * (uint32_t)B + (uint32_t)b;
            const int64_t j = i + dlo + b;
            int32_t sigma = mismatch;
            if (act) sigma = dev_pair(qc, dev_base(bpk, bnb, sb + (uint64_t)j), match, mismatch);
            const int32_t Dg = Hd + sigma;
            int32_t cand;
            uint32_t Sc;
            if (Dg >= E) { cand = Dg; Sc = SD; } else { cand = E; Sc = SE; }
            const int32_t H0 = cand > 0 ? cand : 0;
            // F by max-scan with carry from earlier chunks of this row
            int32_t xv = act ? H0 + goe - ge * (int32_t)b : SW_XNEG;
            uint32_t xs = Sc;
            scan_pair_max(xv, xs, lane);
            int32_t ev = __shfl_up_sync(0xffffffffu, xv, 1);
            uint32_t es = __shfl_up_sync(0xffffffffu, xs, 1);
            // the carry (earlier chunks) wins only when strictly larger
            if (lane == 0) { ev = carry_v; es = carry_s; }
            else if (carry_v > ev) { ev = carry_v; es = carry_s; }
            int32_t last_v = __shfl_sync(0xffffffffu, xv, 31);
            uint32_t last_s = __shfl_sync(0xffffffffu, xs, 31);
            if (last_v >= carry_v) { carry_v = last_v; carry_s = last_s; }
            int32_t F = (ev > SW_XNEG) ? ev + ge * (int32_t)(b - 1) : SW_NEG;
            uint32_t SF = es;
            int32_t H;
            uint32_t SH;
            if (H0 >= F) { H = H0; SH = Sc; } else { H = F; SH = SF; }
            if (act) {
                SwCell c;
                c.H = H; c.E = E; c.SH = SH; c.SE = SE;
                row[b] = c;
                if (H > best) { best = H; bi = i; bj = j; bs = SH; }
            }
            __syncwarp();
        }
    }
    // reduce: highest score, then smallest i, then smallest j
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
            int64_t i0 = I0 + (int64_t)(bs / (uint32_t)B);
            int64_t j0 = i0 + dlo + (int64_t)(bs % (uint32_t)B);
            res.qs = (uint32_t)i0; res.qe = (uint32_t)(bi + 1);
            res.ds = (uint32_t)j0; res.de = (uint32_t)(bj + 1);
            res.score = best;
        }
        out[task] = res;
    }
}

// 32 consecutive bases of a packed sequence starting at a 16-aligned position: 2-bit
// codes (first base most significant) and non-base flags (bit = offset).
struct BaseWin {
    uint64_t p0 = ~0ull, codes = 0;
    uint32_t bad = 0;
    __device__ __forceinline__ void load(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb, uint64_t p) {
        p0 = p & ~15ull;
        const uint64_t w = p0 >> 4;
        codes = ((uint64_t)pk[w] << 32) | pk[w + 1];
        const uint64_t v = p0 >> 5;
        bad = (p0 & 31) ? ((nb[v] >> 16) | (nb[v + 1] << 16)) : nb[v];
    }
    // code of base p (p0 <= p < p0 + 32), 4 for a non-base
    __device__ __forceinline__ uint32_t at(uint64_t p) const {
        const uint32_t o = (uint32_t)(p - p0);
        return ((bad >> o) & 1u) ? 4u : (uint32_t)(codes >> (62 - 2 * o)) & 3u;
    }
};

// 64 consecutive bases [p0, p0 + 64) of a packed sequence (p0 a multiple of 16) that
// slide forward 16 at a time, with the next 16 bases loaded one slide ahead, so a
// warp walking rows rarely waits on memory.  All lanes of a segment hold the same
// window.  Words at or past `end` (the sequence's end) are never read.
struct SegWin {
    uint64_t p0 = 0, hi = 0, lo = 0, bad = 0;  // codes of p0..p0+31 (hi) and p0+32..p0+63 (lo); non-base bits
    uint32_t nxt_pk = 0, nxt_nb = 0;            // the 16 bases after the window (code word, non-base word)
    __device__ __forceinline__ static uint32_t pk_at(const uint32_t *__restrict__ pk, uint64_t x, uint64_t end) {
        return x < end ? pk[x >> 4] : 0u;
    }
    __device__ __forceinline__ static uint32_t nb_at(const uint32_t *__restrict__ nb, uint64_t x, uint64_t end) {
        return x < end ? nb[x >> 5] : 0u;
    }
    __device__ __forceinline__ void prefetch(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb,
                                             uint64_t end) {
        nxt_pk = pk_at(pk, p0 + 64, end);
        nxt_nb = nb_at(nb, p0 + 64, end);
    }
    __device__ __forceinline__ void init(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb, uint64_t p,
                                         uint64_t end) {
        p0 = p & ~15ull;
        hi = ((uint64_t)pk_at(pk, p0, end) << 32) | pk_at(pk, p0 + 16, end);
        lo = ((uint64_t)pk_at(pk, p0 + 32, end) << 32) | pk_at(pk, p0 + 48, end);
        // bit o = base p0 + o; words of 32 bases hold p0 at bit 0 or at bit 16
        if (p0 & 16) {
            bad = ((uint64_t)nb_at(nb, p0, end) >> 16) | ((uint64_t)nb_at(nb, p0 + 16, end) << 16) |
                  ((uint64_t)nb_at(nb, p0 + 48, end) << 48);
        } else {
            bad = (uint64_t)nb_at(nb, p0, end) | ((uint64_t)nb_at(nb, p0 + 32, end) << 32);
        }
        prefetch(pk, nb, end);
    }
    __device__ __forceinline__ void advance(const uint32_t *__restrict__ pk, const uint32_t *__restrict__ nb,
                                            uint64_t end) {
        const uint64_t q = p0 + 64;
        hi = (hi << 32) | (lo >> 32);
        lo = (lo << 32) | nxt_pk;
        bad = (bad >> 16) | ((uint64_t)((nxt_nb >> (q & 16)) & 0xFFFFu) << 48);
        p0 += 16;
        prefetch(pk, nb, end);
    }
    // code of base p (p0 <= p < p0 + 64), 4 for a non-base
    __device__ __forceinline__ uint32_t at(uint64_t p) const {
        const uint32_t o = (uint32_t)(p - p0);
        const uint32_t c = (uint32_t)((o < 32 ? hi : lo) >> (62 - 2 * (o & 31))) & 3u;
        return ((bad >> o) & 1ull) ? 4u : c;
    }
};

// Codes of the bases at offsets o, o + 1, ... of a window from the top of a 64-bit
// word (2 bits each; -31 <= o < 64, offsets outside the window read as 0), and their
// non-base bits from bit 0.
__device__ __forceinline__ uint64_t segwin_codes(const SegWin &wn, int32_t o) {
    if (o < 0) return wn.hi >> (2 * -o);
    if (o == 0) return wn.hi;
    if (o < 32) return (wn.hi << (2 * o)) | (wn.lo >> (64 - 2 * o));
    return wn.lo << (2 * (o - 32));
}
__device__ __forceinline__ uint32_t segwin_bad(const SegWin &wn, int32_t o) {
    return o < 0 ? (uint32_t)(wn.bad << -o) : (uint32_t)(wn.bad >> o);
}

// Code of the base at offset o (0 <= o < 64) of a window, 4 for a non-base.
__device__ __forceinline__ uint32_t segwin_code(const SegWin &wn, uint32_t o) {
    const uint32_t word = o < 32 ? (o < 16 ? (uint32_t)(wn.hi >> 32) : (uint32_t)wn.hi)
                                 : (o < 48 ? (uint32_t)(wn.lo >> 32) : (uint32_t)wn.lo);
    const uint32_t c = (word >> (30 - 2 * (o & 15))) & 3u;
    const uint32_t badw = o < 32 ? (uint32_t)wn.bad : (uint32_t)(wn.bad >> 32);
    return ((badw >> (o & 31)) & 1u) ? 4u : c;
}

// 32 / G HSPs per warp: segment s (lanes sG .. sG + G - 1) aligns its own HSP, lane l of
// the segment owns band offsets K l .. K l + K - 1 and keeps their previous-row states
// in registers.  All segments step through rows together.  The vertical-gap input of
// offset b is offset b + 1 of the previous row (own state, or the next lane's first
// offset); horizontal gaps come from a segmented warp max-scan as in the pair path.
// A cell outside the DP region keeps H = 0 and E = -inf as its state, so the next row
// reads its neighbours without range checks: a neutral neighbour yields only E <= 0 and
// a diagonal from H = 0, neither of which can raise a score (an alignment may begin at
// any cell); a per-row bit mask of the lane's cells in the region masks the stored
// state and the best cell.  Every tracked maximum is a DPX max with its predicate
// (__vibmax_s32: the first operand wins ties), which also selects the start cell.
// Returns with handled = false (and computes nothing) for an HSP whose band exceeds G K
// offsets.
template <int G, int K>
__device__ __forceinline__ void sw_group(bool valid, const DevHsp &h, const uint32_t *__restrict__ qpk,
                                         const uint32_t *__restrict__ qnb, const uint64_t *__restrict__ qstart,
                                         const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                         const uint64_t *__restrict__ seq_start, int32_t match, int32_t mismatch,
                                         int32_t goe, int32_t ge, int32_t w, bool &handled, DevAln &res) {
    const int lane = threadIdx.x & 31, sl = lane % G;
    int64_t I0 = 0, I1 = 0, J0 = 0, J1 = 0, dlo = 0, B = 0;
    uint64_t qb = 0, sb = 0, qend = 0, send = 0;
    if (valid) {
        qb = qstart[h.qi];
        sb = seq_start[h.seq];
        qend = qstart[h.qi + 1];
        send = seq_start[h.seq + 1];
        const int64_t m = (int64_t)(qend - qb), L = (int64_t)(send - sb);
        const int64_t d_s = (int64_t)h.ds - h.qs, d_e = (int64_t)h.de - h.qe;
        dlo = min(d_s, d_e) - w;
        B = max(d_s, d_e) + w - dlo + 1;
        I0 = max((int64_t)0, (int64_t)h.qs - w);
        I1 = min(m, (int64_t)h.qe + w);
        J0 = max((int64_t)0, (int64_t)h.ds - w);
        J1 = min(L, (int64_t)h.de + w);
    }
    handled = valid && B <= G * K && I1 - I0 <= 65535;
    const int32_t rows = handled ? (int32_t)(I1 - I0) : 0;
    const int32_t max_rows = __reduce_max_sync(0xffffffffu, (uint32_t)rows);
    const int32_t jlo = (int32_t)(J0 - I0 - dlo), jhi = (int32_t)(J1 - 1 - I0 - dlo);
    const int32_t Bm1 = (int32_t)B - 1;
    const int32_t b0 = K * sl;
    // per-offset constants: X(b) = H0(b) + cX[k], F(b) = max_{b' < b} X(b') + cF[k]
    int32_t cX[K], cF[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cX[k] = goe - ge * (b0 + k);
        cF[k] = ge * (b0 + k - 1);
    }
    int32_t pH[K], pE[K];
    uint32_t pSH[K], pSE[K];
#pragma unroll
    for (int k = 0; k < K; ++k) { pH[k] = 0; pE[k] = SW_NEG; pSH[k] = 0; pSE[k] = 0; }
    int32_t best = 0;
    uint32_t bpos = 0xFFFFFFFFu, bs = 0;  // best cell: row << 16 | band offset, and its start cell
    // bases: one 64-base window per segment (bands of up to 49 diagonals), else a
    // 32-base window per lane
    constexpr bool SEG = G * K <= 49;
    BaseWin wq, wd;
    SegWin sq, sd;
    if (SEG && handled) {
        sq.init(qpk, qnb, qb + (uint64_t)I0, qend);
        sd.init(bpk, bnb, sb + (uint64_t)max(I0 + dlo, J0), send);
    }
    for (int32_t r = 0; r < max_rows; ++r) {
        const bool seg_on = r < rows;
        const int32_t blo = max(0, jlo - r), bhi = min(Bm1, jhi - r);
        // the lane's offsets b0 + k inside [blo, bhi]
        const int32_t klo = max(blo - b0, 0), khi = min(bhi - b0, K - 1);
        const uint32_t amask = (seg_on && klo <= khi) ? ((2u << khi) - 1u) & ~((1u << klo) - 1u) : 0u;
        const bool lane_on = amask != 0u;
        // previous-row state of offset K (sl + 1) (the next lane's first offset); the last lane's
        // is beyond the band
        int32_t uH = __shfl_down_sync(0xffffffffu, pH[0], 1, G), uE = __shfl_down_sync(0xffffffffu, pE[0], 1, G);
        const uint32_t uSH = __shfl_down_sync(0xffffffffu, pSH[0], 1, G);
        const uint32_t uSE = __shfl_down_sync(0xffffffffu, pSE[0], 1, G);
        if (sl == G - 1) { uH = 0; uE = SW_NEG; }
        uint32_t qc = 4u;
        const uint64_t i = (uint64_t)(I0 + r);
        const uint64_t jb = sb + (uint64_t)((int64_t)i + dlo + b0);  // bank position of offset b0
        if (SEG) {
            if (seg_on) {  // the same in every lane of the segment
                if (qb + i >= sq.p0 + 64) sq.advance(qpk, qnb, qend);
                const uint64_t jhi_pos = sb + (uint64_t)min((int64_t)i + dlo + B - 1, J1 - 1);
                if (jhi_pos >= sd.p0 + 64) sd.advance(bpk, bnb, send);
                if (lane_on) qc = sq.at(qb + i);
            }
        } else if (lane_on) {
            if (i + qb < wq.p0 || i + qb >= wq.p0 + 32) wq.load(qpk, qnb, qb + i);
            qc = wq.at(qb + i);
            const uint64_t jfirst = jb + (uint64_t)max(0, blo - b0), jlast = jb + (uint64_t)min(K - 1, bhi - b0);
            if (jfirst < wd.p0 || jlast >= wd.p0 + 32) wd.load(bpk, bnb, jfirst);
        }
        // the lane's K bank bases (window offsets o0 .. o0 + K - 1; o0 >= -(K - 1))
        uint64_t dcodes = 0;
        uint32_t dbad = 0;
        if (SEG && lane_on) {
            const int32_t o0 = (int32_t)((int64_t)jb - (int64_t)sd.p0);
            dcodes = segwin_codes(sd, o0);
            dbad = segwin_bad(sd, o0);
        }
        // bit k: offset b0 + k pairs two equal bases (the row's query base against the K codes)
        uint32_t dm = 0;
        if (SEG && lane_on && qc < 4u) {
            const uint32_t x = ~((uint32_t)(dcodes >> 32) ^ (qc * 0x55555555u)), eq = x & (x >> 1);
#pragma unroll
            for (int k = 0; k < K; ++k) dm |= ((eq >> (30 - 2 * k)) & 1u) << k;
            dm &= ~dbad;
        }
        const uint32_t rowbase = (uint32_t)r << 16;
        int32_t H0[K], E[K], X[K];
        uint32_t C[K], SE[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            // vertical gap from offset b + 1 of the previous row: open wins ties
            const int32_t vH = k + 1 < K ? pH[k + 1] : uH, vE = k + 1 < K ? pE[k + 1] : uE;
            const uint32_t vSH = k + 1 < K ? pSH[k + 1] : uSH, vSE = k + 1 < K ? pSE[k + 1] : uSE;
            bool po;
            E[k] = __vibmax_s32(vH + goe, vE + ge, &po);
            SE[k] = po ? vSH : vSE;
            // diagonal: from the previous row's H, or a start here
            const int32_t Hd = pH[k];
            const uint32_t SD = Hd > 0 ? pSH[k] : rowbase | (uint32_t)(b0 + k);
            bool same;
            if (SEG) {
                same = (dm >> k) & 1u;
            } else {
                const uint32_t d = ((amask >> k) & 1u) ? wd.at(jb + k) : 4u;  // the window covers the active cells only
                same = qc < 4u && d == qc;
            }
            const int32_t Dg = Hd + (same ? match : mismatch);
            // diagonal over E on ties
            bool pd;
            const int32_t cv = __vibmax_s32(Dg, E[k], &pd);
            C[k] = pd ? SD : SE[k];
            H0[k] = max(cv, 0);
            X[k] = H0[k] + cX[k];
        }
        // lane aggregate of X (later offsets win ties), then the segmented scan over lanes
        int32_t xv = X[0];
        uint32_t xs = C[0];
#pragma unroll
        for (int k = 1; k < K; ++k) {
            bool p;
            xv = __vibmax_s32(X[k], xv, &p);
            xs = p ? C[k] : xs;
        }
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            const int32_t ov = __shfl_up_sync(0xffffffffu, xv, o, G);
            const uint32_t os = __shfl_up_sync(0xffffffffu, xs, o, G);
            bool p;
            xv = __vibmax_s32(xv, sl >= o ? ov : SW_XNEG, &p);
            xs = p ? xs : os;
        }
        int32_t ev = __shfl_up_sync(0xffffffffu, xv, 1, G);
        uint32_t es = __shfl_up_sync(0xffffffffu, xs, 1, G);
        if (sl == 0) { ev = SW_XNEG; es = 0; }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            // H0 over F on ties
            bool ph;
            const int32_t Hv = __vibmax_s32(H0[k], ev + cF[k], &ph);
            const uint32_t S = ph ? C[k] : es;
            bool px;
            ev = __vibmax_s32(X[k], ev, &px);
            es = px ? C[k] : es;
            const bool act = (amask >> k) & 1u;
            const int32_t Hm = act ? Hv : 0;
            if (Hm > best) { best = Hm; bpos = rowbase | (uint32_t)(b0 + k); bs = S; }
            pH[k] = Hm; pE[k] = act ? E[k] : SW_NEG; pSH[k] = S; pSE[k] = SE[k];
        }
    }
    // segment reduction: highest score, then smallest row, then smallest offset (smallest j)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const int32_t ob = __shfl_down_sync(0xffffffffu, best, o, G);
        const uint32_t op = __shfl_down_sync(0xffffffffu, bpos, o, G);
        const uint32_t os = __shfl_down_sync(0xffffffffu, bs, o, G);
        if (ob > best || (ob == best && op < bpos)) { best = ob; bpos = op; bs = os; }
    }
    res.qi = h.qi; res.seq = h.seq; res.qs = res.qe = res.ds = res.de = 0; res.score = 0; res.pad = 0;
    if (handled && best > 0) {
        const int64_t bi = I0 + (int64_t)(bpos >> 16), bj = bi + dlo + (int64_t)(bpos & 0xFFFFu);
        const int64_t i0 = I0 + (int64_t)(bs >> 16), j0 = i0 + dlo + (int64_t)(bs & 0xFFFFu);
        res.qs = (uint32_t)i0; res.qe = (uint32_t)(bi + 1);
        res.ds = (uint32_t)j0; res.de = (uint32_t)(bj + 1);
        res.score = best;
    }
}

// One HSP with a band of at most 64 diagonals on anti-diagonal wavefronts, for the
// longest alignments, whose row-by-row chains would otherwise bound the kernel's time.
// Cell (r, b) (row I0 + r, band offset b) lies on wavefront t = 2r + b; its diagonal
// input (r - 1, b) is on t - 2, its vertical input (r - 1, b + 1) and horizontal input
// (r, b - 1) on t - 1.  Lane l owns offsets 2l and 2l + 1 and computes one of them per
// wavefront (offset 2l on even t, 2l + 1 on odd t), so each wavefront takes one
// shuffle step and a short chain of operations instead of a row's scan.  Each cell
// follows the sequential recurrence with its tie rules: E and F open on ties, the
// diagonal beats E, H0 beats F; F extends from the left cell's H0 (as the row scan
// does).  The best cell is the highest score, then the smallest row, then the
// smallest offset.  Start cells are (row - I0) * B + offset.
struct WaveCell {
    int32_t H, E, H0, F;
    uint32_t SH, SE, C, SF;
};

__device__ __forceinline__ void sw_wave(const DevHsp &h, const uint32_t *__restrict__ qpk,
                                        const uint32_t *__restrict__ qnb, const uint64_t *__restrict__ qstart,
                                        const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                        const uint64_t *__restrict__ seq_start, int32_t match, int32_t mismatch,
                                        int32_t goe, int32_t ge, int32_t w, DevAln &res) {
    const int lane = threadIdx.x & 31;
    const uint64_t qb = qstart[h.qi], sb = seq_start[h.seq], qend = qstart[h.qi + 1], send = seq_start[h.seq + 1];
    const int64_t m = (int64_t)(qend - qb), L = (int64_t)(send - sb);
    const int64_t d_s = (int64_t)h.ds - h.qs, d_e = (int64_t)h.de - h.qe;
    const int64_t dlo = min(d_s, d_e) - w;
    const int32_t B = (int32_t)(max(d_s, d_e) + w - dlo + 1);
    const int64_t I0 = max((int64_t)0, (int64_t)h.qs - w), I1 = min(m, (int64_t)h.qe + w);
    const int64_t J0 = max((int64_t)0, (int64_t)h.ds - w), J1 = min(L, (int64_t)h.de + w);
    const int32_t rows = (int32_t)max(I1 - I0, (int64_t)0);
    const int32_t jlo = (int32_t)(J0 - I0 - dlo), jhi = (int32_t)(J1 - 1 - I0 - dlo);
    // rows r where offset e is a cell of the window: max(0, jlo - e) <= r <= min(rows - 1, jhi - e)
    const int32_t b0 = 2 * lane, b1 = 2 * lane + 1;
    auto lo_of = [&](int32_t e) { return (e >= 0 && e < B) ? max(0, jlo - e) : INT32_MAX; };
    auto hi_of = [&](int32_t e) { return (e >= 0 && e < B) ? min(rows - 1, jhi - e) : -1; };
    const int32_t lo_m = lo_of(b0 - 1), hi_m = hi_of(b0 - 1), lo_0 = lo_of(b0), hi_0 = hi_of(b0);
    const int32_t lo_1 = lo_of(b1), hi_1 = hi_of(b1), lo_2 = lo_of(b1 + 1), hi_2 = hi_of(b1 + 1);
    WaveCell c0, c1;  // the lane's last cells at offsets 2l and 2l + 1
    c0.H = c1.H = 0; c0.E = c1.E = SW_NEG; c0.H0 = c1.H0 = 0; c0.F = c1.F = SW_NEG;
    c0.SH = c1.SH = c0.SE = c1.SE = c0.C = c1.C = c0.SF = c1.SF = 0;
    bool v0 = false, v1 = false;  // cells (r - 1, 2l) and (r - 1, 2l + 1) were in the window
    int32_t best = 0, br = INT32_MAX, bb = INT32_MAX;
    uint32_t bs = 0;
    SegWin sq, sd;
    sq.init(qpk, qnb, qb + (uint64_t)I0, qend);
    sd.init(bpk, bnb, sb + (uint64_t)max(I0 + dlo, J0), send);
    // window offsets of this lane's bases at iteration k = t / 2 (row r = k - l): query
    // base I0 + r, bank base I0 + dlo + r + 2l (offset 2l; 2l + 1 is the next one)
    int32_t oq = (int32_t)((int64_t)(qb + (uint64_t)I0) - (int64_t)sq.p0) - lane;
    int32_t od = (int32_t)((int64_t)sb + I0 + dlo - (int64_t)sd.p0) + lane;
    int32_t qmax = (int32_t)((int64_t)(qb + (uint64_t)I0) - (int64_t)sq.p0);  // lane 0's query offset
    // last bank offset the wavefront pair t, t + 1 reads: I0 + dlo + (t + B) / 2, at most J1 - 1
    const int64_t dmax0 = (int64_t)sb + I0 + dlo - (int64_t)sd.p0;
    const int64_t dcap = (int64_t)sb + J1 - 1 - (int64_t)sd.p0;
    int32_t dshift = 0;  // 16 x the bank window's advances
    uint32_t rB = (uint32_t)(-lane) * (uint32_t)B;  // r * B (start cells)
    const int32_t T = rows > 0 ? 2 * rows + B - 2 : 0;  // wavefronts 0 .. T - 1
    for (int32_t t = 0, r = -lane; t < T; t += 2, ++r, ++oq, ++od, ++qmax, rB += (uint32_t)B) {
        if (qmax >= 64) { sq.advance(qpk, qnb, qend); oq -= 16; qmax -= 16; }
        if (min(dmax0 + (t + B) / 2, dcap) - dshift >= 64) { sd.advance(bpk, bnb, send); od -= 16; dshift += 16; }
        const uint32_t qc = (r >= 0 && r < rows) ? segwin_code(sq, (uint32_t)oq) : 4u;
        // even wavefront t: cell (r, 2l); left (r, 2l - 1) is lane l - 1's, from wavefront t - 1
        {
            const int32_t lH0 = __shfl_up_sync(0xffffffffu, c1.H0, 1), lF = __shfl_up_sync(0xffffffffu, c1.F, 1);
            const uint32_t lC = __shfl_up_sync(0xffffffffu, c1.C, 1), lSF = __shfl_up_sync(0xffffffffu, c1.SF, 1);
            const bool cv = r >= lo_0 && r <= hi_0;
            int32_t E = SW_NEG;
            uint32_t SE = 0;
            if (cv && v1) {  // up-right (r - 1, 2l + 1): own, from wavefront t - 1
                const int32_t eo = c1.H + goe, ee = c1.E + ge;
                if (eo >= ee) { E = eo; SE = c1.SH; } else { E = ee; SE = c1.SE; }
            }
            const int32_t Hd = (cv && v0) ? c0.H : 0;
            const uint32_t SD = Hd > 0 ? c0.SH : rB + (uint32_t)b0;
            const int32_t sc = cv ? dev_pair(qc, segwin_code(sd, (uint32_t)od), match, mismatch) : mismatch;
            const int32_t Dg = Hd + sc;
            int32_t cand;
            uint32_t C;
            if (Dg >= E) { cand = Dg; C = SD; } else { cand = E; C = SE; }
            const int32_t H0 = cand > 0 ? cand : 0;
            int32_t F = SW_NEG;
            uint32_t SF = 0;
            if (cv && r >= lo_m && r <= hi_m) {
                const int32_t fo = lH0 + goe, fe = lF + ge;
                if (fo >= fe) { F = fo; SF = lC; } else { F = fe; SF = lSF; }
            }
            int32_t H;
            uint32_t SH;
            if (H0 >= F) { H = H0; SH = C; } else { H = F; SH = SF; }
            // cells of one lane come in row-major order: the first maximum wins
            if (cv && H > best) { best = H; br = r; bb = b0; bs = SH; }
            c0.H = H; c0.E = E; c0.H0 = H0; c0.F = F; c0.SH = SH; c0.SE = SE; c0.C = C; c0.SF = SF;
            v0 = cv;
        }
        // odd wavefront t + 1: cell (r, 2l + 1); up-right (r - 1, 2l + 2) is lane l + 1's, from wavefront t
        {
            const int32_t uH = __shfl_down_sync(0xffffffffu, c0.H, 1), uE = __shfl_down_sync(0xffffffffu, c0.E, 1);
            const uint32_t uSH = __shfl_down_sync(0xffffffffu, c0.SH, 1), uSE = __shfl_down_sync(0xffffffffu, c0.SE, 1);
            const bool cv = r >= lo_1 && r <= hi_1;
            int32_t E = SW_NEG;
            uint32_t SE = 0;
            if (cv && r - 1 >= lo_2 && r - 1 <= hi_2) {
                const int32_t eo = uH + goe, ee = uE + ge;
                if (eo >= ee) { E = eo; SE = uSH; } else { E = ee; SE = uSE; }
            }
            const int32_t Hd = (cv && v1) ? c1.H : 0;
            const uint32_t SD = Hd > 0 ? c1.SH : rB + (uint32_t)b1;
            const int32_t sc = cv ? dev_pair(qc, segwin_code(sd, (uint32_t)od + 1u), match, mismatch) : mismatch;
            const int32_t Dg = Hd + sc;
            int32_t cand;
            uint32_t C;
            if (Dg >= E) { cand = Dg; C = SD; } else { cand = E; C = SE; }
            const int32_t H0 = cand > 0 ? cand : 0;
            int32_t F = SW_NEG;
            uint32_t SF = 0;
            if (cv && v0) {  // left (r, 2l): own, just computed
                const int32_t fo = c0.H0 + goe, fe = c0.F + ge;
                if (fo >= fe) { F = fo; SF = c0.C; } else { F = fe; SF = c0.SF; }
            }
            int32_t H;
            uint32_t SH;
            if (H0 >= F) { H = H0; SH = C; } else { H = F; SH = SF; }
            if (cv && H > best) { best = H; br = r; bb = b1; bs = SH; }
            c1.H = H; c1.E = E; c1.H0 = H0; c1.F = F; c1.SH = SH; c1.SE = SE; c1.C = C; c1.SF = SF;
            v1 = cv;
        }
    }
    // highest score, then smallest row, then smallest offset
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t ob = __shfl_down_sync(0xffffffffu, best, o);
        const int32_t orr = __shfl_down_sync(0xffffffffu, br, o), obb = __shfl_down_sync(0xffffffffu, bb, o);
        const uint32_t os = __shfl_down_sync(0xffffffffu, bs, o);
        if (ob > best || (ob == best && (orr < br || (orr == br && obb < bb)))) { best = ob; br = orr; bb = obb; bs = os; }
    }
    res.qi = h.qi; res.seq = h.seq; res.qs = res.qe = res.ds = res.de = 0; res.score = 0; res.pad = 0;
    if (best > 0) {
        const int64_t bi = I0 + br, bj = bi + dlo + bb;
        const int64_t i0 = I0 + (int64_t)(bs / (uint32_t)B), j0 = i0 + dlo + (int64_t)(bs % (uint32_t)B);
        res.qs = (uint32_t)i0; res.qe = (uint32_t)(bi + 1);
        res.ds = (uint32_t)j0; res.de = (uint32_t)(bj + 1);
        res.score = best;
    }
}

// Warps take 32 / SWG_G selected HSPs at a time; each segment of SWG_G lanes aligns one
// whose band fits SWG_G x SWG_K offsets, and the whole warp then aligns the others one by
// one (pair or strip path).
// SWG_G lanes per HSP (32 / SWG_G HSPs per warp), SWG_K band offsets per lane: <8, 5>
// (bands of up to 40 diagonals, the default), <16, 3> (48) or <32, 2> (64).
template <int SWG_G, int SWG_K>
__global__ void __launch_bounds__(128, 1) k_banded_sw(const DevHsp *__restrict__ sel, uint32_t n,
                                                   const uint64_t *__restrict__ strip_off, SwCell *__restrict__ strips,
                                                   const uint32_t *__restrict__ qpk, const uint32_t *__restrict__ qnb,
                                                   const uint64_t *__restrict__ qstart,
                                                   const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                                   const uint64_t *__restrict__ seq_start, int32_t match,
                                                   int32_t mismatch, int32_t go, int32_t ge, int32_t w,
                                                   uint32_t *__restrict__ next_task, const uint64_t *__restrict__ order,
                                                   uint32_t *__restrict__ wide, uint32_t *__restrict__ wide_count,
                                                   const uint32_t *__restrict__ n_long, uint32_t *__restrict__ next_long,
                                                   DevAln *__restrict__ out, uint32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31, seg = lane / SWG_G;
    constexpr int NG = 32 / SWG_G;
    // the first n_long tasks of the order (the longest alignments): one warp each on wavefronts
    const uint32_t nl = *n_long;
    for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(next_long, 1u);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= nl) break;
        const uint32_t task = (uint32_t)order[j];
        const DevHsp h = sel[task];
        if (dev_band(h, w) > 64) {
            if (lane == 0) wide[atomicAdd(wide_count, 1u)] = task;
            continue;
        }
        DevAln res;
        sw_wave(h, qpk, qnb, qstart, bpk, bnb, seq_start, match, mismatch, go + ge, ge, w, res);
        if (lane == 0) out[task] = res;
    }
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(next_task, (uint32_t)NG);
        base = __shfl_sync(0xffffffffu, base, 0) + nl;
        if (base >= n) return;
        const bool valid = base + seg < n;
        const uint32_t task = valid ? (uint32_t)order[base + seg] : 0u;  // longest alignments first
        DevHsp h{};
        if (valid) h = sel[task];
        bool handled = false;
        DevAln res;
        sw_group<SWG_G, SWG_K>(valid, h, qpk, qnb, qstart, bpk, bnb, seq_start, match, mismatch, go + ge, ge, w,
                               handled, res);
        if (handled && lane % SWG_G == 0) out[task] = res;
        // wider bands: one HSP at a time with the whole warp
        uint32_t rest = __ballot_sync(0xffffffffu, valid && !handled && lane % SWG_G == 0);
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            const uint32_t t2 = (uint32_t)order[base + (uint32_t)(src / SWG_G)];
            if (dev_band(sel[t2], w) > 64) {  // wide bands: k_banded_sw_wide
                if (lane == 0) wide[atomicAdd(wide_count, 1u)] = t2;
                continue;
            }
            sw_task_warp<false>(sel, t2, strip_off, strips, qpk, qnb, qstart, bpk, bnb, seq_start, match, mismatch, go,
                                ge, w, out, status);
            __syncwarp();
        }
    }
}

// Bands wider than 64 diagonals, one HSP per warp: up to 32 x SWW_K offsets with the
// row states in registers (the grouped path over the whole warp), wider ones on the
// strip path.  A kernel of its own, so that its registers do not limit the main
// alignment kernel.
constexpr int SWW_K = 9;
__global__ void __launch_bounds__(128) k_banded_sw_wide(const DevHsp *__restrict__ sel, const uint32_t *__restrict__ wide,
                                                        const uint32_t *__restrict__ wide_count,
                                                        uint32_t *__restrict__ next, const uint64_t *__restrict__ strip_off,
                                                        SwCell *__restrict__ strips, const uint32_t *__restrict__ qpk,
                                                        const uint32_t *__restrict__ qnb, const uint64_t *__restrict__ qstart,
                                                        const uint32_t *__restrict__ bpk, const uint32_t *__restrict__ bnb,
                                                        const uint64_t *__restrict__ seq_start, int32_t match,
                                                        int32_t mismatch, int32_t go, int32_t ge, int32_t w,
                                                        DevAln *__restrict__ out, uint32_t *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const uint32_t n = *wide_count;
    for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(next, 1u);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= n) return;
        const uint32_t task = wide[j];
        const DevHsp h = sel[task];
        bool handled = false;
        DevAln res;
        sw_group<32, SWW_K>(true, h, qpk, qnb, qstart, bpk, bnb, seq_start, match, mismatch, go + ge, ge, w, handled,
                            res);
        if (handled) {
            if (lane == 0) out[task] = res;
        } else {
            sw_task_warp<true>(sel, task, strip_off, strips, qpk, qnb, qstart, bpk, bnb, seq_start, match, mismatch,
                               go, ge, w, out, status);
        }
        __syncwarp();
    }
}

// Preparation of the alignment phase, per selected HSP:
// - the strip length of its band (B + 1), and the band area (DP-window rows x B, the cells
//   the alignment kernels evaluate) summed into cells[0] (bands of at most 64 diagonals) or
//   cells[1] (wider bands);
// - its alignment-order key (65535 - DP-window rows) << 32 | task, so that an ascending sort
//   on bits 32..47 hands out the longest alignments first (they bound the kernel's time) and
//   groups alignments of similar length; alignments of at least long_rows rows are counted
//   in *n_long (they sort first).
__global__ void k_sw_prepare(const DevHsp *__restrict__ h, uint32_t n, int32_t w, const uint64_t *__restrict__ qstart,
                             uint32_t *__restrict__ B, unsigned long long *__restrict__ cells, uint32_t long_rows,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ n_long) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < n;
    int64_t rows = 0;
    if (in) {
        const DevHsp x = h[i];
        const int64_t d_s = (int64_t)x.ds - x.qs, d_e = (int64_t)x.de - x.qe;
        const int64_t b = (max(d_s, d_e) + w) - (min(d_s, d_e) - w) + 1;
        B[i] = (uint32_t)min(b + 1, (int64_t)65537);  // +1: the strip is read at b + 1
        const int64_t m = (int64_t)(qstart[x.qi + 1] - qstart[x.qi]);
        rows = min(m, (int64_t)x.qe + w) - max((int64_t)0, (int64_t)x.qs - w);
        if (rows > 0) atomicAdd(cells + (b > 64 ? 1 : 0), (unsigned long long)(rows * b));
        const int64_t r = rows < 0 ? 0 : (rows > 65535 ? 65535 : rows);
        keys[i] = ((uint64_t)(65535 - (uint32_t)r) << 32) | i;
    }
    const uint32_t lng = __ballot_sync(0xffffffffu, in && rows >= (int64_t)min(long_rows, 65535u));
    if ((threadIdx.x & 31) == 0 && lng) atomicAdd(n_long, (uint32_t)__popc(lng));
}

// ------------------------------------------------------ a13: ranking --
__global__ void k_dup_flags(const DevAln *__restrict__ a, uint32_t n, uint32_t *__restrict__ flag) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DevAln x = a[i];
    bool keep = x.score > 0;
    if (keep && i > 0) {
        const DevAln y = a[i - 1];
        if (y.qi == x.qi && y.seq == x.seq && y.qs == x.qs && y.qe == x.qe && y.ds == x.ds && y.de == x.de)
            keep = false;
    }
    flag[i] = keep ? 1u : 0u;
}

__global__ void k_finalize(const DevAln *__restrict__ a, uint32_t n, const uint32_t *__restrict__ first,
                           const uint64_t *__restrict__ qstart, double n_bank, double lambda, double K,
                           double max_e, gn_hit *__restrict__ out, uint32_t *__restrict__ flag) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DevAln x = a[i];
    double m = (double)(qstart[x.qi + 1] - qstart[x.qi]);
    gn_hit h;
    h.query = x.qi; h.seq = x.seq; h.q_start = x.qs; h.q_end = x.qe; h.db_start = x.ds; h.db_end = x.de;
    h.score = x.score;
    h.rank = i - first[x.qi];
    h.evalue = K * m * n_bank * exp(-lambda * (double)x.score);
    h.bits = (lambda * (double)x.score - log(K)) / log(2.0);
    out[i] = h;
    flag[i] = (h.evalue <= max_e) ? 1u : 0u;
}


// Per-query ranking (alignments of a query are contiguous and at most RQ_CAP): one
// CTA per query sorts record indices in shared memory with a bitonic network - first
// by (seq, q_start, q_end, db_start, db_end, score desc) to drop records that repeat
// an earlier one's sequence and ranges (and records with score <= 0), then by
// (score desc, seq, q_start, db_start, q_end, db_end) - and writes the ranked hits
// with e-value and bit score at the query's input offset.
constexpr int RQ_CAP = 1024;

__device__ __forceinline__ bool rq_less_dedupe(const DevAln &a, const DevAln &b) {
    if (a.seq != b.seq) return a.seq < b.seq;
    if (a.qs != b.qs) return a.qs < b.qs;
    if (a.qe != b.qe) return a.qe < b.qe;
    if (a.ds != b.ds) return a.ds < b.ds;
    if (a.de != b.de) return a.de < b.de;
    return a.score > b.score;
}

__device__ __forceinline__ bool rq_less_rank(const DevAln &a, const DevAln &b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.seq != b.seq) return a.seq < b.seq;
    if (a.qs != b.qs) return a.qs < b.qs;
    if (a.ds != b.ds) return a.ds < b.ds;
    if (a.qe != b.qe) return a.qe < b.qe;
    return a.de < b.de;
}

template <int MODE>  // 0: dedupe order, 1: rank order (dropped records last)
__device__ void rq_bitonic(uint16_t *idx, const DevAln *rec, const uint8_t *keep, uint32_t P) {
    for (uint32_t k2 = 2; k2 <= P; k2 <<= 1) {
        for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint16_t a = idx[i], c = idx[ixj];
                    bool a_gt_c;  // a sorts after c
                    if (a == 0xFFFFu) a_gt_c = c != 0xFFFFu;
                    else if (c == 0xFFFFu) a_gt_c = false;
                    else if (MODE == 1 && keep[a] != keep[c]) a_gt_c = !keep[a];
                    else a_gt_c = MODE == 0 ? rq_less_dedupe(rec[c], rec[a]) : rq_less_rank(rec[c], rec[a]);
                    const bool up = (i & k2) == 0;
                    if (a_gt_c == up) { idx[i] = c; idx[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_rank_query(const DevAln *__restrict__ aln, const uint32_t *__restrict__ qrange,
                                                    uint32_t nq, const uint64_t *__restrict__ qstart, double n_bank,
                                                    double lambda, double K, double max_e, gn_hit *__restrict__ out,
                                                    uint32_t *__restrict__ qcount) {
    __shared__ DevAln rec[RQ_CAP];
    __shared__ uint16_t idx[RQ_CAP];
    __shared__ uint8_t keep[RQ_CAP];
    __shared__ uint32_t nk_s, ne_s;
    for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
        const uint32_t start = qrange[2 * q], n = qrange[2 * q + 1] - start;
        if (n == 0) {
            if (threadIdx.x == 0) qcount[q] = 0;
            continue;
        }
        uint32_t P = 1;
        while (P < n) P <<= 1;
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
            if (i < n) rec[i] = aln[start + i];
            idx[i] = i < n ? (uint16_t)i : (uint16_t)0xFFFFu;
        }
        if (threadIdx.x == 0) { nk_s = 0; ne_s = 0; }
        __syncthreads();
        rq_bitonic<0>(idx, rec, keep, P);
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
            const DevAln &a = rec[idx[k]];
            bool kk = a.score > 0;
            if (kk && k > 0) {
                const DevAln &b = rec[idx[k - 1]];
                kk = !(a.seq == b.seq && a.qs == b.qs && a.qe == b.qe && a.ds == b.ds && a.de == b.de);
            }
            keep[idx[k]] = kk ? 1 : 0;
            if (kk) atomicAdd(&nk_s, 1u);
        }
        __syncthreads();
        rq_bitonic<1>(idx, rec, keep, P);
        const uint32_t nk = nk_s;
        const double m = (double)(qstart[rec[0].qi + 1] - qstart[rec[0].qi]);
        for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
            const DevAln &x = rec[idx[k]];
            gn_hit h;
            h.query = x.qi; h.seq = x.seq; h.q_start = x.qs; h.q_end = x.qe; h.db_start = x.ds; h.db_end = x.de;
            h.score = x.score;
            h.rank = k;
            h.evalue = K * m * n_bank * exp(-lambda * (double)x.score);
            h.bits = (lambda * (double)x.score - log(K)) / log(2.0);
            // e-values rise as scores fall, so the cut keeps a prefix of the ranking
            if (h.evalue <= max_e) {
                out[start + k] = h;
                atomicAdd(&ne_s, 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) qcount[q] = ne_s;
        __syncthreads();
    }
}

__global__ void k_query_ranges(const DevAln *__restrict__ a, uint32_t n, uint32_t *__restrict__ qrange) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t q = a[i].qi;
    if (i == 0 || a[i - 1].qi != q) qrange[2 * q] = i;
    if (i == n - 1 || a[i + 1].qi != q) qrange[2 * q + 1] = i + 1;
}

__global__ void k_gather_ranked(const gn_hit *__restrict__ in, const uint32_t *__restrict__ qrange,
                                const uint64_t *__restrict__ qoff, uint32_t nq, gn_hit *__restrict__ out) {
    for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
        const uint32_t start = qrange[2 * q];
        const uint64_t o = qoff[q], c = qoff[q + 1] - o;
        for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) out[o + k] = in[start + k];
    }
}

// ------------------------------------------------------------ compaction --
__global__ void k_scatter_flagged(const uint32_t *__restrict__ in, int W, const uint32_t *__restrict__ flags,
                                  const uint64_t *__restrict__ pos, uint32_t n, uint32_t *__restrict__ out) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * W) return;
    uint32_t i = (uint32_t)(t / W), w = (uint32_t)(t % W);
    if (flags[i]) out[pos[i] * W + w] = in[t];
}

uint32_t compact_records(const uint32_t *in, int W, const uint32_t *flags, uint32_t n, uint32_t *out,
                         DeviceArena &arena, cudaStream_t s) {
    if (n == 0) return 0;
    uint64_t *pos = arena.alloc_n<uint64_t>(n + 1);
    void *scr = arena.alloc(scan_scratch_bytes(n));
    exclusive_scan_u32(flags, pos, n, scr, s);
    uint64_t tot = (uint64_t)n * W;
    GN_LAUNCH("k_scatter_flagged", n, s,
              k_scatter_flagged<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(in, W, flags, pos, n, out));
    uint64_t cnt = 0;
    GN_CUDA(cudaMemcpyAsync(&cnt, pos + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    return (uint32_t)cnt;
}

// ---------------------------------------------------------------- driver --
namespace {
struct PhaseTimer {
    cudaStream_t s;
    std::vector<std::pair<const char *, cudaEvent_t>> marks;
    explicit PhaseTimer(cudaStream_t st) : s(st) {}
    void mark(const char *name) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, s);
        marks.emplace_back(name, e);
    }
    void finish(std::vector<std::pair<const char *, float>> &out) {
        out.clear();
        for (size_t i = 1; i < marks.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second);
            out.emplace_back(marks[i].first, ms);
        }
    }
    ~PhaseTimer() {
        for (auto &m : marks) cudaEventDestroy(m.second);
    }
};

template <class T>
std::vector<T> to_host(const T *d, size_t n, cudaStream_t s) {
    std::vector<T> h(n);
    if (n) {
        GN_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
        GN_CUDA(cudaStreamSynchronize(s));
    }
    return h;
}

unsigned blocks_for(uint64_t n, unsigned t = 256) { return (unsigned)std::max<uint64_t>(1, (n + t - 1) / t); }

// Lets the kernels with a per-call dynamic shared-memory size use up to the device's opt-in
// maximum.  Set once per device: concurrent searches (serving threads) launch with different
// sizes, and a per-call attribute change by one thread could undercut another's launch.
void allow_max_smem(int device) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64 || done[device]) return;
    int optin = 0;
    GN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    auto allow = [&](const void *fn) {  // the opt-in maximum less the kernel's static shared memory
        cudaFuncAttributes fa;
        GN_CUDA(cudaFuncGetAttributes(&fa, fn));
        GN_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
    };
    allow(reinterpret_cast<const void *>(k_bucket_fill<0, 0>));
    allow(reinterpret_cast<const void *>(k_bucket_fill<19, 17>));
    allow(reinterpret_cast<const void *>(k_bucket_group_warp));
    done[device] = true;
}
}  // namespace

// Both strands: query i of the input becomes query 2i (the bases as given) and query
// 2i + 1 (its reverse complement) of the output, back to back.  Complement: A <-> T,
// C <-> G in either case, U (read as T) -> A; any other byte is a non-base and stays.
__device__ __forceinline__ uint8_t dev_complement(uint8_t c) {
    switch (c) {
        case 'A': return 'T'; case 'T': return 'A'; case 'U': return 'A';
        case 'C': return 'G'; case 'G': return 'C';
        case 'a': return 't'; case 't': return 'a'; case 'u': return 'a';
        case 'c': return 'g'; case 'g': return 'c';
        default: return c;
    }
}
__global__ void k_both_strands(const uint8_t *__restrict__ in, const uint64_t *__restrict__ qstart, uint32_t nq,
                               uint64_t M, uint8_t *__restrict__ out) {
    const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= M) return;
    const uint32_t i = dev_upper_index(qstart, nq + 1, x);
    const uint64_t s0 = qstart[i], m = qstart[i + 1] - s0, p = x - s0;
    const uint8_t c = in[x];
    out[2 * s0 + p] = c;
    out[2 * s0 + m + (m - 1 - p)] = dev_complement(c);
}

void both_strands(const uint8_t *qbases_dev, const std::vector<uint64_t> &qstart_h, DeviceArena &arena,
                  cudaStream_t s, const uint8_t **out_bases, std::vector<uint64_t> &out_start) {
    const uint32_t nq = (uint32_t)(qstart_h.size() - 1);
    const uint64_t M = qstart_h[nq];
    out_start.assign(2ull * nq + 1, 0);
    for (uint32_t i = 0; i < nq; ++i) {
        const uint64_t m = qstart_h[i + 1] - qstart_h[i];
        out_start[2 * i + 1] = 2 * qstart_h[i] + m;
        out_start[2 * i + 2] = 2 * qstart_h[i] + 2 * m;
    }
    uint8_t *d = arena.alloc_n<uint8_t>(2 * M);
    uint64_t *qs = arena.alloc_n<uint64_t>(nq + 1);
    GN_CUDA(cudaMemcpyAsync(qs, qstart_h.data(), 8ull * (nq + 1), cudaMemcpyHostToDevice, s));
    if (M) GN_LAUNCH("k_both_strands", M, s, k_both_strands<<<blocks_for(M), 256, 0, s>>>(qbases_dev, qs, nq, M, d));
    *out_bases = d;
}

void search(gn_index *ix, const uint8_t *qbases_dev, const std::vector<uint64_t> &qstart_h, const SearchOptions &o,
            cudaStream_t s, gn_results *res) {
    const uint32_t nq = (uint32_t)(qstart_h.size() - 1);
    const uint64_t M = qstart_h[nq];
    const int k = ix->span;  // HSPs end k bases after their last seed (the seed's span)
    const gn_params &p = o.p;
    const gn_scoring &sc = o.sc;
    const bool keep = (p.flags & GN_FLAG_KEEP_STAGES) != 0;
    const bool keep_hits = (p.flags & GN_FLAG_KEEP_HITS) != 0;
    res->n_queries = nq;
    res->has_stages = keep;
    PhaseTimer timer(s);
    timer.mark("start");
    KernelTimer ktimer;
    struct TimerScope {
        KernelTimer *prev;
        explicit TimerScope(KernelTimer *t) : prev(g_ktimer) { g_ktimer = t; }
        ~TimerScope() { g_ktimer = prev; }
    };
    TimerScope tscope((p.flags & GN_FLAG_TIME_KERNELS) ? &ktimer : nullptr);
    DeviceArena arena(s);
    // bounded device-side waits (the scans' look-back) record a timeout here
    uint32_t *wait_status = arena.alloc_n<uint32_t>(1);
    GN_CUDA(cudaMemsetAsync(wait_status, 0, 4, s));
    WaitStatusScope wscope(wait_status);
#ifdef GN_CHECKS
    uint32_t *check_bits = nullptr;  // the failed device-side checks of this search
    GN_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&check_bits), g_check_bits));
    GN_CUDA(cudaMemsetAsync(check_bits, 0, 4, s));
#endif

    // a5: pack queries, code every offset, list lengths
    Packed qp;
    qp.pk = arena.alloc_n<uint32_t>(Packed::pk_words(M));
    qp.nb = arena.alloc_n<uint32_t>(Packed::nb_words(M));
    pack_bases(qbases_dev, M, qp, s);
    uint64_t *qstart_d = arena.alloc_n<uint64_t>(nq + 1);
    GN_CUDA(cudaMemcpyAsync(qstart_d, qstart_h.data(), sizeof(uint64_t) * (nq + 1), cudaMemcpyHostToDevice, s));

    // The seed phases (a5-a8) run on the queries themselves, or, when a query is longer
    // than MAX_QUERY_LEN, on segments: every query of at most MAX_QUERY_LEN bases is one
    // segment, a longer one is cut into segments of MAX_QUERY_LEN bases SEG_STEP apart
    // (neighbours share SEG_OVERLAP bases; the last one ends with the query).  Every
    // chain of hits at most D offsets apart then has each pair of consecutive hits inside
    // one segment (D + span <= SEG_OVERLAP), so the chain is the union of its pieces in
    // the segments, and pieces of one chain share a hit.  The pieces are emitted whatever
    // their length, mapped back onto the query and joined after a8 (k_stitch_sweep),
    // which then applies min_hsp_len.
    std::vector<uint64_t> seg_start{0}, seg_off;  // per segment: start in the segment batch, offset in its query
    std::vector<uint32_t> seg_parent;
    bool segmented = false;
    uint64_t max_qlen = 0;
    for (uint32_t i = 0; i < nq; ++i) {
        const uint64_t m = qstart_h[i + 1] - qstart_h[i];
        max_qlen = std::max(max_qlen, m);
        for (uint64_t o = 0;; o += SEG_STEP) {
            const uint64_t len = std::min<uint64_t>(MAX_QUERY_LEN, m - o);
            seg_parent.push_back(i);
            seg_off.push_back(o);
            seg_start.push_back(seg_start.back() + len);
            if (o + MAX_QUERY_LEN >= m) break;
            segmented = true;
        }
    }
    GN_REQUIRE(seg_parent.size() <= MAX_QUERIES, GN_ETOOBIG, "more than 65,536 query segments in one call");
    if (segmented) {
        GN_REQUIRE(p.max_hit_distance + (uint32_t)k <= SEG_OVERLAP, GN_EINVAL,
                   "queries over 65,535 bases need max_hit_distance + seed span <= 8,192");
        GN_REQUIRE(!(p.flags & (GN_FLAG_KEEP_STAGES | GN_FLAG_KEEP_HITS)), GN_EINVAL,
                   "stage outputs are not kept for queries over 65,535 bases");
        GN_REQUIRE(ix->max_seq_len < (1ull << 32) - (1ull << 24), GN_ETOOBIG,
                   "queries over 65,535 bases need bank sequences shorter than 2^32 - 2^24 bases");
    }
    const uint32_t hnq = segmented ? (uint32_t)seg_parent.size() : nq;
    const std::vector<uint64_t> &hstart_h = segmented ? seg_start : qstart_h;
    const uint64_t HM = hstart_h[hnq];
    const uint32_t hit_min_len = segmented ? 1u : p.min_hsp_len;
    Packed hqp = qp;
    uint64_t *hstart_d = qstart_d;
    uint32_t *seg_parent_d = nullptr;
    uint64_t *seg_off_d = nullptr;
    if (segmented) {
        hstart_d = arena.alloc_n<uint64_t>(hnq + 1);
        seg_off_d = arena.alloc_n<uint64_t>(hnq);
        seg_parent_d = arena.alloc_n<uint32_t>(hnq);
        GN_CUDA(cudaMemcpyAsync(hstart_d, seg_start.data(), sizeof(uint64_t) * (hnq + 1), cudaMemcpyHostToDevice, s));
        GN_CUDA(cudaMemcpyAsync(seg_off_d, seg_off.data(), sizeof(uint64_t) * hnq, cudaMemcpyHostToDevice, s));
        GN_CUDA(cudaMemcpyAsync(seg_parent_d, seg_parent.data(), sizeof(uint32_t) * hnq, cudaMemcpyHostToDevice, s));
        uint8_t *sb = arena.alloc_n<uint8_t>(HM);
        GN_LAUNCH("k_segment_bases", HM, s,
                  k_segment_bases<<<hnq, 256, 0, s>>>(qbases_dev, qstart_d, seg_parent_d, seg_off_d, hstart_d, sb));
        hqp.pk = arena.alloc_n<uint32_t>(Packed::pk_words(HM));
        hqp.nb = arena.alloc_n<uint32_t>(Packed::nb_words(HM));
        pack_bases(sb, HM, hqp, s);
    }
    uint32_t *codes = arena.alloc_n<uint32_t>(HM);
    uint32_t *qinfo = arena.alloc_n<uint32_t>(HM);
    uint32_t *cnt = arena.alloc_n<uint32_t>(HM);
    uint32_t *src = arena.alloc_n<uint32_t>(HM);
    uint64_t *hoff = arena.alloc_n<uint64_t>(HM + 1);
    if (HM) {
        GN_LAUNCH("k_query_codes", HM, s,
                  k_query_codes<<<blocks_for(HM), 256, 0, s>>>(hstart_d, hnq, HM, hqp.pk, hqp.nb, seed_shape(ix), ix->off_d, codes, qinfo,
                                                              cnt, src));
    }
    {
        void *scr = arena.alloc(scan_scratch_bytes(HM));
        exclusive_scan_u32(cnt, hoff, HM, scr, s);
    }
    // hit offsets at query boundaries -> per-query hit counts (chunk plan)
    uint64_t *hq_d = arena.alloc_n<uint64_t>(hnq + 1);
    GN_LAUNCH("k_gather_u64", hnq + 1, s,
              k_gather_u64<<<blocks_for(hnq + 1), 256, 0, s>>>(hoff, hstart_d, hnq + 1, hq_d));
    std::vector<uint64_t> hq = to_host(hq_d, hnq + 1, s);
    GN_REQUIRE(!o.max_hit_bytes || hq[hnq] * HIT_BYTES <= o.max_hit_bytes, GN_ETOOBIG,
               "the query alone exceeds the server's memory budget");
    timer.mark("query_codes");
    if (keep) {
        res->st_hit_counts.resize(hnq);
        for (uint32_t i = 0; i < hnq; ++i) res->st_hit_counts[i] = hq[i + 1] - hq[i];
    }

    // a6-a8 per chunk of queries whose hits fit the budget
    size_t free_b = 0, total_b = 0;
    GN_CUDA(cudaMemGetInfo(&free_b, &total_b));
    // bytes per hit of a chunk: hit keys and their ping-pong buffer on the sort path, or the
    // fixed-capacity buckets (up to ~22 B per hit without the repeat filter) and spill lists
    uint64_t mem_for_hits = (uint64_t)(free_b * 0.55);
    if (o.mem_cap) mem_for_hits = std::min(mem_for_hits, o.mem_cap);
    // (a query chunk holds < 2^32 hits: the fill kernel indexes a tile's hits in 32 bits)
    uint64_t hit_budget = std::min<uint64_t>(0xFFFFFFFFull, std::max<uint64_t>(1ull << 20, mem_for_hits / HIT_BYTES));
    if (const char *e = getenv("GN_MAX_CHUNK_HITS")) {  // smaller chunks (exercises the multi-chunk path)
        uint64_t v = strtoull(e, nullptr, 10);
        if (v) hit_budget = std::min<uint64_t>(v, 0xFFFFFFFFull);
    }
    const uint64_t gbits_max = (uint64_t)bits_for(ix->n_bases + QBIAS);
    const uint32_t max_chunk_q = (uint32_t)std::min<uint64_t>(MAX_QUERIES, 1ull << std::min<uint64_t>(48 - gbits_max, 31));

    uint32_t hsp_cap = (uint32_t)std::min<uint64_t>(0xFFFFFFFFull, std::max<uint64_t>(1u << 16, hq[hnq] / 128));
    DevHsp *hsp = arena.alloc_n<DevHsp>(hsp_cap);
    uint32_t n_hsp = 0;
    uint32_t *counter = arena.alloc_n<uint32_t>(4);
    uint32_t *status = arena.alloc_n<uint32_t>(1);
    GN_CUDA(cudaMemsetAsync(status, 0, 4, s));
    std::vector<uint32_t> hits_q;

    uint32_t qa = 0;
    while (qa < hnq) {
        uint32_t qb = qa + 1;
        while (qb < hnq && qb - qa < max_chunk_q && hq[qb + 1] - hq[qa] <= hit_budget) ++qb;
        const uint64_t xa = hstart_h[qa], xb = hstart_h[qb];
        const uint64_t ha = hq[qa], Hc = hq[qb] - hq[qa];
        GN_REQUIRE(Hc < (1ull << 32), GN_ETOOBIG, "a query has 2^32 seed hits or more");
        if (Hc > 0) {
            const int qbits = bits_for(qb - qa - 1);
            const int gbits = (int)gbits_max;
            const uint32_t nqc = qb - qa;
            DeviceArena carena(s);
            // appends HSPs through `launch(out, room)`, growing the HSP buffer and relaunching on overflow
            auto emit = [&](auto launch) {
                for (int attempt = 0; attempt < 3; ++attempt) {
                    GN_CUDA(cudaMemsetAsync(counter, 0, 4, s));
                    launch(hsp + n_hsp, hsp_cap - n_hsp);
                    uint32_t got = 0;
                    GN_CUDA(cudaMemcpyAsync(&got, counter, 4, cudaMemcpyDeviceToHost, s));
                    GN_CUDA(cudaStreamSynchronize(s));
                    if (n_hsp + (uint64_t)got <= hsp_cap) {
                        n_hsp += got;
                        return;
                    }
                    uint64_t need = (uint64_t)n_hsp + got;
                    GN_REQUIRE(need < (1ull << 32), GN_ETOOBIG, "more than 2^32 HSPs in one call");
                    uint32_t ncap = (uint32_t)std::min<uint64_t>(0xFFFFFFFFull,
                                                                 std::max<uint64_t>(need + need / 4, 2ull * hsp_cap));
                    DevHsp *nh = arena.alloc_n<DevHsp>(ncap);
                    if (n_hsp) GN_CUDA(cudaMemcpyAsync(nh, hsp, sizeof(DevHsp) * n_hsp, cudaMemcpyDeviceToDevice, s));
                    hsp = nh;
                    hsp_cap = ncap;
                    GN_CUDA(cudaMemsetAsync(status, 0, 4, s));
                }
                throw Error{GN_EINTERNAL, "HSP buffer growth did not converge"};
            };
            // global path: gather every hit, LSD radix sort by diagonal key, merge sorted runs
            auto sort_path = [&](uint64_t *keys, uint64_t *keys_alt, uint64_t n, int lo_bit, const RadixTag &tag) {
                void *rs = carena.alloc(radix_scratch_bytes(n));
                bool fl = radix_sort(keys, keys_alt, nullptr, nullptr, n, lo_bit, 16 + qbits + gbits, rs, s, tag);
                uint64_t *sorted = fl ? keys_alt : keys;
                timer.mark("hit_sort");
                emit([&](DevHsp *o, uint32_t room) {
                    uint64_t threads = std::min<uint64_t>(n, (uint64_t)num_sms() * 2048);
                    GN_LAUNCH("k_hit_merge", n, s,
                              k_hit_merge<<<blocks_for(threads), 256, 0, s>>>(sorted, n, qbits, qa, k,
                                                                             p.max_hit_distance, hit_min_len,
                                                                             seq_map(ix), o, counter, room, status));
                });
                return sorted;
            };
            const char *grouping = getenv("GN_HIT_GROUPING");
            const bool bucketed = !keep_hits && !(grouping && strcmp(grouping, "sort") == 0);
            if (!bucketed) {
                uint64_t *keys = carena.alloc_n<uint64_t>(Hc);
                uint64_t *keys_alt = carena.alloc_n<uint64_t>(Hc);
                uint64_t gwarps = std::min<uint64_t>((xb - xa + 31) / 32, (uint64_t)num_sms() * 64);
                GN_LAUNCH("k_seed_gather", Hc, s,
                          k_seed_gather<<<blocks_for(gwarps * 32), 256, 0, s>>>(codes, qinfo, hoff, xa, xb, ha,
                                                                               ix->off_d, ix->post_d, qa, qbits,
                                                                               keys));
                timer.mark("seed_gather");
                uint64_t *sorted = sort_path(keys, keys_alt, Hc, 16 + qbits, TAG_HIT_SORT);
                if (keep_hits) {
                    uint32_t *quad = carena.alloc_n<uint32_t>(4 * Hc);
                    GN_LAUNCH("k_decode_hits", Hc, s,
                              k_decode_hits<<<blocks_for(Hc), 256, 0, s>>>(sorted, Hc, qbits, qa, ix->seq_start_d,
                                                                           ix->n_seqs, quad));
                    std::vector<uint32_t> hh = to_host(quad, 4 * Hc, s);
                    hits_q.insert(hits_q.end(), hh.begin(), hh.end());
                }
            } else {
                // bucket plan: 2^lg buckets per query, about `target` raw hits each
                const int singles = p.min_hsp_len <= (uint32_t)k ? 1 : 0;
                const char *fenv = getenv("GN_TILE_FILTER");
                const int filter = (!singles && p.max_hit_distance <= (uint32_t)BT_MAX_D &&
                                    !(fenv && strcmp(fenv, "0") == 0)) ? 1 : 0;
                // 512-thread tiles of about 50,000 hits: 512 offsets at ~88 hits per offset (stride 11 on
                // a 4 Gbp bank), fewer where lists are long (small strides), up to 1,024 where they are
                // short; 2^19-bit "seen" and 2^17-bit "seen twice" bitmaps (two tiles per SM)
                const double per_offset = (double)Hc / (double)std::max<uint64_t>(1, xb - xa);
                const double tile_hits = ix->tuning.tile_hits ? (double)ix->tuning.tile_hits : 50000.0;
                int tpos = 32;
                while (tpos < 1024 && tpos * 2 * per_offset <= tile_hits * 1.5) tpos *= 2;
                // a small search (one query, a few) gets smaller tiles, so that its hits are spread
                // over the SMs instead of filling one or two tiles one after the other
                while (tpos > 32 && (xb - xa + tpos - 1) / tpos < 4ull * (uint64_t)num_sms()) tpos /= 2;
                int fthreads = ix->tuning.fill_threads == 256 ? 256 : 512;
                if (const char *e = getenv("GN_FILL_THREADS")) fthreads = atoi(e) >= 512 ? 512 : 256;
                // two 512-thread tiles or four 256-thread tiles per SM
                int fbits = fthreads == 512 ? 19 : 18, fbits2 = fthreads == 512 ? 17 : 16;
                if (const char *e = getenv("GN_TILE_POS")) tpos = std::max(32, std::min(4096, atoi(e)));
                if (const char *e = getenv("GN_TILE_FBITS")) fbits = std::max(12, std::min(19, atoi(e)));
                if (const char *e = getenv("GN_TILE_FBITS2")) fbits2 = std::max(12, std::min(19, atoi(e)));
                // the filter keeps about 2 % of the hits: buckets of about 4,096 raw hits hold about 80 kept
                // hits, most of them within the grouping warps' 256 candidates; capacity 1,024
                uint32_t target = filter ? (ix->tuning.bucket_target ? ix->tuning.bucket_target : 4096) : 512, bcap = 1024;
                if (const char *e = getenv("GN_BUCKET_TARGET")) target = std::max(64, std::min(65536, atoi(e)));
                if (const char *e = getenv("GN_BUCKET_CAP")) {  // small buckets (exercises the spill path)
                    bcap = (uint32_t)std::max(8ul, std::min(65536ul, strtoul(e, nullptr, 10)));
                    target = std::max<uint32_t>(2, bcap / 2);
                }
                const bool fixed_cap = getenv("GN_BUCKET_CAP") != nullptr;
                std::vector<uint32_t> bbase(nqc + 1), bshift(nqc);
                const int min_lg = std::max(0, gbits - 31);
                uint32_t NB = 0;
                uint32_t *d_bbase = carena.alloc_n<uint32_t>(nqc + 1);
                uint32_t *d_bshift = carena.alloc_n<uint32_t>(nqc);
                uint32_t *bcount = nullptr;
                uint64_t *bkeys = nullptr;
                uint16_t *bq = nullptr;
                // 2^lg buckets per query, about `target` raw hits each
                auto plan = [&](uint64_t target) {
                    uint64_t nb64 = 0;
                    for (uint32_t i = 0; i < nqc; ++i) {
                        const uint64_t hi = hq[qa + i + 1] - hq[qa + i];
                        const uint64_t want = (hi + target - 1) / target;
                        int lg = 0;
                        while ((1ull << lg) < want) ++lg;
                        lg = std::min(std::max(lg, min_lg), gbits);
                        bshift[i] = (uint32_t)(gbits - lg);
                        bbase[i] = (uint32_t)nb64;
                        nb64 += 1ull << lg;
                        GN_REQUIRE(nb64 < (1ull << 32), GN_ETOOBIG, "too many hit buckets in one chunk");
                    }
                    bbase[nqc] = (uint32_t)nb64;
                    NB = (uint32_t)nb64;
                    GN_CUDA(cudaMemcpyAsync(d_bbase, bbase.data(), 4 * (nqc + 1), cudaMemcpyHostToDevice, s));
                    GN_CUDA(cudaMemcpyAsync(d_bshift, bshift.data(), 4 * nqc, cudaMemcpyHostToDevice, s));
                };
                auto alloc_buckets = [&]() {
                    bcount = carena.alloc_n<uint32_t>(NB);
                    bkeys = carena.alloc_n<uint64_t>((uint64_t)NB * bcap);
                    bq = carena.alloc_n<uint16_t>(NB);
                };
                plan(target);
                unsigned long long *spill_count = reinterpret_cast<unsigned long long *>(carena.alloc_n<uint64_t>(1));
                uint64_t spill_room = std::max<uint64_t>(1u << 16, Hc / 32);
                uint64_t min_room = 0;  // GN_SPILL_ROOM: small first rooms (exercises the reruns)
                if (const char *e = getenv("GN_SPILL_ROOM")) min_room = std::max<uint64_t>(1, strtoull(e, nullptr, 10));
                if (min_room) spill_room = min_room;
                uint64_t *spill = carena.alloc_n<uint64_t>(spill_room);
                const uint64_t tiles = (xb - xa + tpos - 1) / tpos;
                // the kept-hit stage gets what the SM's shared memory leaves for two 512-thread (or four
                // 256-thread) tiles per SM after the filters and the table, at least 256 hits
                uint32_t stage_cap = 256;
                {
                    const uint32_t halo = filter ? p.max_hit_distance : 0u;
                    int per_sm = 0, reserved = 0;
                    GN_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ix->device));
                    GN_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ix->device));
                    const int64_t room = (int64_t)per_sm / (fthreads == 512 ? 2 : 4) - reserved - 512 -
                                         (int64_t)bucket_fill_smem(tpos, halo, filter, fbits, fbits2, 0);
                    if (room > 256 * BF_STAGE_BYTES)
                        stage_cap = (uint32_t)std::min<int64_t>(8192, room / BF_STAGE_BYTES) & ~31u;
                }
                const size_t bf_smem = bucket_fill_smem(tpos, filter ? p.max_hit_distance : 0u, filter, fbits, fbits2,
                                                        stage_cap);
                auto fill_kernel = (fbits == 19 && fbits2 == 17) ? k_bucket_fill<19, 17> : k_bucket_fill<0, 0>;
                allow_max_smem(ix->device);
                int focc = 0;
                GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&focc, fill_kernel, fthreads, bf_smem));
                const unsigned fgrid = (unsigned)std::max<uint64_t>(
                    1, std::min<uint64_t>(tiles, (uint64_t)num_sms() * std::max(focc, 1) * 4));
                unsigned long long n_spill = 0, n_kept = 0;
                // kept hits, core hits (sampling), tile counter
                unsigned long long *kept_total = reinterpret_cast<unsigned long long *>(carena.alloc_n<uint64_t>(3));
                // Keep rate of the repeat filter, measured on a sample of tiles (no placement): the plan
                // above assumes the stride-11 rate; where far more hits are kept (small strides, where
                // overlapping k-mers put most hits next to another on their diagonal) the buckets are
                // planned smaller.
                // With a keep rate above a quarter, 256-entry buckets of about 128 kept hits are planned:
                // the grouping warps take every such bucket whole.
                auto plan_for_keep = [&](double keep, uint32_t &t_new, uint32_t &cap_new) {
                    if (keep > 0.25) {
                        cap_new = 256;
                        t_new = (uint32_t)std::max(64.0, 128.0 / keep);
                    } else {
                        cap_new = bcap;
                        t_new = (uint32_t)std::max(64.0, std::min((double)target, bcap / 2.0 / keep));
                    }
                };
                if (filter && !fixed_cap && !getenv("GN_BUCKET_TARGET") && ix->t < 8) {
                    const uint32_t tile_step = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(256, tiles / 256));
                    const uint64_t stiles = (tiles + tile_step - 1) / tile_step;
                    unsigned long long got[2] = {0, 0};
                    GN_CUDA(cudaMemsetAsync(kept_total, 0, 24, s));
                    GN_LAUNCH("k_bucket_fill_sample", Hc / tile_step, s,
                              fill_kernel<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(stiles, fgrid)), fthreads,
                                            bf_smem, s>>>(
                                  qinfo, src, hoff, xa, xb, ix->post_d, qa, d_bbase, d_bshift, nullptr, nullptr, bcap,
                                  nullptr, nullptr, 0ull, qbits, filter, p.max_hit_distance, tpos, fbits, fbits2,
                                  kept_total, tile_step, 1, stage_cap, NB, post_alloc_entries(ix->n_postings) / 4));
                    GN_CUDA(cudaMemcpyAsync(got, kept_total, 16, cudaMemcpyDeviceToHost, s));
                    GN_CUDA(cudaStreamSynchronize(s));
                    if (got[1]) {
                        uint32_t t_new = target, cap_new = bcap;
                        plan_for_keep(std::max(1e-6, (double)got[0] / (double)got[1]), t_new, cap_new);
                        if (t_new != target || cap_new != bcap) {
                            target = t_new;
                            bcap = cap_new;
                            plan(target);
                        }
                    }
                }
                alloc_buckets();
                // Which of two colliding keys the filter keeps depends on arrival order, so the spill
                // count varies a little between runs: a rerun gets room with a margin, and the loop
                // ends on the run whose spills all fit.
                auto run_fill = [&]() {
                    for (int attempt = 0;; ++attempt) {
                        GN_CUDA(cudaMemsetAsync(bcount, 0, 4ull * NB, s));
                        GN_CUDA(cudaMemsetAsync(spill_count, 0, 8, s));
                        GN_CUDA(cudaMemsetAsync(kept_total, 0, 24, s));
                        GN_LAUNCH("k_bucket_fill", Hc, s,
                                  fill_kernel<<<fgrid, fthreads, bf_smem, s>>>(
                                      qinfo, src, hoff, xa, xb, ix->post_d, qa, d_bbase, d_bshift, bcount, bkeys, bcap,
                                      spill, spill_count, (unsigned long long)spill_room, qbits, filter,
                                      p.max_hit_distance, tpos, fbits, fbits2, kept_total, 1u, 0, stage_cap, NB,
                                      post_alloc_entries(ix->n_postings) / 4));
                        GN_CUDA(cudaMemcpyAsync(&n_spill, spill_count, 8, cudaMemcpyDeviceToHost, s));
                        GN_CUDA(cudaMemcpyAsync(&n_kept, kept_total, 8, cudaMemcpyDeviceToHost, s));
                        GN_CUDA(cudaStreamSynchronize(s));
                        if (n_spill <= spill_room) break;
                        GN_REQUIRE(attempt < 3, GN_EINTERNAL, "hit-bucket spill sizing did not converge");
                        spill_room = n_spill + n_spill / 8 + 1024;
                        spill = carena.alloc_n<uint64_t>(spill_room);
                    }
                };
                run_fill();
                // The plan assumes the stride-11 keep rate of the repeat filter.  Where far more hits
                // are kept (small strides: overlapping k-mers put most hits next to another on their
                // diagonal) the buckets overflow; plan again from the measured keep rate, once.
                if (!fixed_cap && n_kept && n_spill > std::max<unsigned long long>(1u << 16, n_kept / 32)) {
                    uint32_t t_new = target, cap_new = bcap;
                    plan_for_keep((double)n_kept / (double)Hc, t_new, cap_new);
                    if (t_new * 4 < target * 3 || cap_new != bcap) {
                        target = t_new;
                        bcap = cap_new;
                        plan(target);
                        alloc_buckets();
                        run_fill();
                    }
                }
                GN_LAUNCH("k_bucket_query", NB, s, k_bucket_query<<<nqc, 256, 0, s>>>(d_bbase, nqc, NB, bq));
                timer.mark("bucket_fill");
                // group each bucket; buckets with too many candidates are appended to the spill list too
                const size_t smem = (size_t)BGW_WARPS * (2 * BGW_BITS / 8 + BGW_CAND * 8 + BGW_CAND / 8);

                int occ = 0;
                GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bucket_group_warp, BGW_WARPS * 32, smem));
                const unsigned ggrid = (unsigned)std::max<uint64_t>(
                    1, std::min<uint64_t>((NB + BGW_WARPS - 1) / BGW_WARPS, (uint64_t)num_sms() * std::max(occ, 1)));
                const uint64_t spilled_fill = n_spill;
                uint64_t group_room = min_room ? min_room : std::max<uint64_t>(1u << 16, Hc / 16);
                uint64_t *gsp = carena.alloc_n<uint64_t>(spilled_fill + group_room);
                if (spilled_fill)
                    GN_CUDA(cudaMemcpyAsync(gsp, spill, 8 * spilled_fill, cudaMemcpyDeviceToDevice, s));
                unsigned long long n_ovf = 0;
                unsigned long long *ovf_count = spill_count;
                uint32_t *big = carena.alloc_n<uint32_t>(NB);  // buckets for the block-level grouping
                uint32_t *big_count = carena.alloc_n<uint32_t>(1);
                uint32_t n_big = 0;
                for (int attempt = 0;; ++attempt) {
                    const uint32_t hsp_before = n_hsp;
                    emit([&](DevHsp *o, uint32_t room) {
                        GN_CUDA(cudaMemsetAsync(ovf_count, 0, 8, s));
                        GN_CUDA(cudaMemsetAsync(counter + 1, 0, 4, s));
                        GN_CUDA(cudaMemsetAsync(big_count, 0, 4, s));
                        GN_LAUNCH("k_bucket_group", n_kept, s,
                                  k_bucket_group_warp<<<ggrid, BGW_WARPS * 32, smem, s>>>(
                                      bkeys, bcount, bcap, NB, bq, qa, qbits, k, p.max_hit_distance, hit_min_len,
                                      singles, seq_map(ix), o, counter, room, gsp + spilled_fill,
                                      (unsigned long long)group_room, ovf_count, status, counter + 1, big,
                                      big_count));
                        // read back with the HSP count, in emit's one synchronisation
                        GN_CUDA(cudaMemcpyAsync(&n_ovf, ovf_count, 8, cudaMemcpyDeviceToHost, s));
                        GN_CUDA(cudaMemcpyAsync(&n_big, big_count, 4, cudaMemcpyDeviceToHost, s));
                    });
                    if (n_ovf <= group_room) break;
                    GN_REQUIRE(attempt < 3, GN_EINTERNAL, "hit-bucket overflow sizing did not converge");
                    n_hsp = hsp_before;  // the rerun emits this chunk's bucket HSPs again
                    group_room = n_ovf + n_ovf / 8 + 1024;
                    uint64_t *ng = carena.alloc_n<uint64_t>(spilled_fill + group_room);
                    if (spilled_fill)
                        GN_CUDA(cudaMemcpyAsync(ng, spill, 8 * spilled_fill, cudaMemcpyDeviceToDevice, s));
                    gsp = ng;
                    GN_CUDA(cudaMemsetAsync(status, 0, 4, s));
                }
                // buckets with more candidates than a warp holds: a block each
                int bocc = 0;
                if (n_big)
                    GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bocc, k_bucket_group_block, 256, 0));
                const unsigned bgrid =
                    (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(n_big, (uint64_t)num_sms() * std::max(bocc, 1)));
                if (n_big) emit([&](DevHsp *o, uint32_t room) {
                    GN_LAUNCH("k_bucket_group_block", n_big, s,
                              k_bucket_group_block<<<bgrid, 256, 0, s>>>(
                                  bkeys, bcount, bcap, bq, big, big_count, qa, k, p.max_hit_distance, hit_min_len,
                                  singles, seq_map(ix), o, counter, room, status));
                });
                timer.mark("bucket_group");
                const uint64_t n_sp = spilled_fill + n_ovf;
                if (n_sp) sort_path(gsp, carena.alloc_n<uint64_t>(n_sp), n_sp, 0, TAG_HIT_SORT);
            }
            timer.mark("hit_merge");
        }
        qa = qb;
    }
    const int qib = bits_for(nq ? nq - 1 : 0);
    const int seqb = bits_for(ix->n_seqs ? ix->n_seqs - 1 : 0);
    const int posb = bits_for(ix->max_seq_len);
    const int qposb = std::max(16, bits_for(max_qlen));
    if (segmented && n_hsp) {
        // pieces onto their queries, then one chain per run of pieces sharing seeds
        GN_LAUNCH("k_segment_map", n_hsp, s,
                  k_segment_map<<<blocks_for(n_hsp), 256, 0, s>>>(hsp, n_hsp, seg_parent_d, seg_off_d));
        uint32_t *perm = arena.alloc_n<uint32_t>(n_hsp);
        sort_records(reinterpret_cast<const uint32_t *>(hsp), HSP_WORDS, n_hsp,
                     {{W_QI, qib, false}, {W_SEQ, seqb, false}, {W_LEN, 32, false}, {W_QS, qposb, false}},
                     perm, arena, s);
        DevHsp *srt = arena.alloc_n<DevHsp>(n_hsp);
        gather_records(reinterpret_cast<const uint32_t *>(hsp), HSP_WORDS, perm, n_hsp,
                       reinterpret_cast<uint32_t *>(srt), s);
        DevHsp *chains = arena.alloc_n<DevHsp>(n_hsp);
        uint32_t *flag = arena.alloc_n<uint32_t>(n_hsp);
        GN_LAUNCH("k_stitch_sweep", n_hsp, s,
                  k_stitch_sweep<<<blocks_for(n_hsp), 256, 0, s>>>(srt, n_hsp, (uint32_t)k, p.min_hsp_len, chains,
                                                                  flag));
        DevHsp *joined = arena.alloc_n<DevHsp>(n_hsp);
        n_hsp = compact_records(reinterpret_cast<const uint32_t *>(chains), HSP_WORDS, flag, n_hsp,
                                reinterpret_cast<uint32_t *>(joined), arena, s);
        hsp = joined;
        timer.mark("stitch");
    }
    if (keep_hits) res->st_hits.swap(hits_q);
    if (keep) {
        std::vector<DevHsp> v = to_host(hsp, n_hsp, s);
        res->st_hsp.resize(n_hsp);
        if (n_hsp) memcpy(res->st_hsp.data(), v.data(), sizeof(DevHsp) * n_hsp);
    }

    // a9: extension
    if (n_hsp) {
        // resident warps only, taking 32-HSP groups from a counter
        uint32_t *next_group = arena.alloc_n<uint32_t>(1);
        GN_CUDA(cudaMemsetAsync(next_group, 0, 4, s));
        int xocc = 0;
        GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&xocc, k_xdrop, 256, 0));
        const uint64_t xwarps =
            std::min<uint64_t>((n_hsp + 31) / 32, (uint64_t)num_sms() * std::max(xocc, 1) * 8);
        // steps a lane walks alone before the warp takes the walk over (GN_XDROP_LANE_STEPS overrides)
        uint32_t lim = 64;
        if (const char *e = getenv("GN_XDROP_LANE_STEPS")) lim = (uint32_t)std::max(0l, strtol(e, nullptr, 10));
        GN_LAUNCH("k_xdrop", n_hsp, s,
                  k_xdrop<<<blocks_for(xwarps * 32, 256), 256, 0, s>>>(hsp, n_hsp, qp.pk, qp.nb, qstart_d,
                                                                      ix->bank.pk, ix->bank.nb, ix->seq_start_d,
                                                                      sc.match, sc.mismatch, p.xdrop, nq, ix->n_seqs,
                                                                      lim, next_group));
    }
    timer.mark("xdrop_extend");
    if (keep) {
        std::vector<DevHsp> v = to_host(hsp, n_hsp, s);
        res->st_ext.resize(n_hsp);
        if (n_hsp) memcpy(res->st_ext.data(), v.data(), sizeof(DevHsp) * n_hsp);
    }

    // a10: merge overlapped HSPs
    uint32_t n_mg = 0;
    DevHsp *merged = arena.alloc_n<DevHsp>(n_hsp);
    if (n_hsp) {
        uint32_t *perm = arena.alloc_n<uint32_t>(n_hsp);
        // (qi, seq, qs) order; the sweep takes the records of one qs by (ds, qe)
        sort_records(reinterpret_cast<const uint32_t *>(hsp), HSP_WORDS, n_hsp,
                     {{W_QI, qib, false}, {W_SEQ, seqb, false}, {W_QS, qposb, false}}, perm, arena, s);
        DevHsp *srt = arena.alloc_n<DevHsp>(n_hsp);
        gather_records(reinterpret_cast<const uint32_t *>(hsp), HSP_WORDS, perm, n_hsp,
                       reinterpret_cast<uint32_t *>(srt), s);
        DevHsp *boxes = arena.alloc_n<DevHsp>(n_hsp);
        uint32_t *flag = arena.alloc_n<uint32_t>(n_hsp);
        GN_LAUNCH("k_overlap_sweep", n_hsp, s,
                  k_overlap_sweep<<<blocks_for(n_hsp), 256, 0, s>>>(srt, n_hsp, boxes, flag));
        n_mg = compact_records(reinterpret_cast<const uint32_t *>(boxes), HSP_WORDS, flag, n_hsp,
                               reinterpret_cast<uint32_t *>(merged), arena, s);
    }
    timer.mark("overlap_merge");
    if (keep) {
        std::vector<DevHsp> v = to_host(merged, n_mg, s);
        res->st_merged.resize(n_mg);
        if (n_mg) memcpy(res->st_merged.data(), v.data(), sizeof(DevHsp) * n_mg);
    }

    // a11: longest first, at most max_alignments per query
    uint32_t n_sel = 0;
    DevHsp *sel = arena.alloc_n<DevHsp>(n_mg);
    uint32_t *first = arena.alloc_n<uint32_t>(nq);
    const char *senv = getenv("GN_SELECT_PATH");
    const bool per_query_select = p.max_alignments > 0 && p.max_alignments <= (uint32_t)SQ_CAP &&
                                  max_qlen <= 65535 && !(senv && strcmp(senv, "sort") == 0);
    if (n_mg && per_query_select) {
        uint32_t *qb = arena.alloc_n<uint32_t>(nq + 1);
        uint32_t *cnt = arena.alloc_n<uint32_t>(nq);
        GN_LAUNCH("k_query_bounds", nq + 1, s,
                  k_query_bounds<<<blocks_for(nq + 1), 256, 0, s>>>(merged, n_mg, nq, qb, p.max_alignments, cnt));
        uint64_t *qo = arena.alloc_n<uint64_t>(nq + 1);
        void *scr = arena.alloc(scan_scratch_bytes(nq));
        exclusive_scan_u32(cnt, qo, nq, scr, s);
        uint64_t tot = 0;
        GN_CUDA(cudaMemcpyAsync(&tot, qo + nq, 8, cudaMemcpyDeviceToHost, s));
        GN_LAUNCH("k_select_query", n_mg, s,
                  k_select_query<<<nq, SQ_THREADS, 0, s>>>(merged, qb, qo, p.max_alignments, sel));
        GN_CUDA(cudaStreamSynchronize(s));
        n_sel = (uint32_t)tot;
    } else if (n_mg) {
        uint32_t *perm = arena.alloc_n<uint32_t>(n_mg);
        sort_records(reinterpret_cast<const uint32_t *>(merged), HSP_WORDS, n_mg,
                     {{W_QI, qib, false}, {W_LEN, qposb, true}, {W_SEQ, seqb, false}, {W_QS, qposb, false},
                      {W_DS, posb, false}, {W_QE, qposb, false}, {W_DE, posb, false}},
                     perm, arena, s);
        DevHsp *srt = arena.alloc_n<DevHsp>(n_mg);
        gather_records(reinterpret_cast<const uint32_t *>(merged), HSP_WORDS, perm, n_mg,
                       reinterpret_cast<uint32_t *>(srt), s);
        GN_LAUNCH("k_first_of_query", 0, s,
                  k_first_of_query<<<blocks_for(n_mg), 256, 0, s>>>(reinterpret_cast<const uint32_t *>(srt), HSP_WORDS, n_mg, first));
        uint32_t *flag = arena.alloc_n<uint32_t>(n_mg);
        GN_LAUNCH("k_select_flags", n_mg, s,
                  k_select_flags<<<blocks_for(n_mg), 256, 0, s>>>(srt, n_mg, first, p.max_alignments, flag));
        n_sel = compact_records(reinterpret_cast<const uint32_t *>(srt), HSP_WORDS, flag, n_mg,
                                reinterpret_cast<uint32_t *>(sel), arena, s);
    }
    timer.mark("select");
    if (keep) {
        std::vector<DevHsp> v = to_host(sel, n_sel, s);
        res->st_sel.resize(n_sel);
        if (n_sel) memcpy(res->st_sel.data(), v.data(), sizeof(DevHsp) * n_sel);
    }

    // a12: banded Smith-Waterman
    DevAln *aln = arena.alloc_n<DevAln>(n_sel);
    if (n_sel) {
        uint32_t *B = arena.alloc_n<uint32_t>(n_sel);
        uint64_t *soff = arena.alloc_n<uint64_t>(n_sel + 1);
        unsigned long long *dp_cells = reinterpret_cast<unsigned long long *>(arena.alloc_n<uint64_t>(2));
        GN_CUDA(cudaMemsetAsync(dp_cells, 0, 16, s));
        uint64_t *okeys = arena.alloc_n<uint64_t>(n_sel), *okeys_alt = arena.alloc_n<uint64_t>(n_sel);
        // alignments of at least sw_long rows go to the wavefront path (their rows would
        // bound the kernel's time on the grouped path)
        uint32_t sw_long = ix->tuning.sw_wave_rows ? ix->tuning.sw_wave_rows : 512;
        if (const char *e = getenv("GN_SW_LONG_ROWS")) sw_long = (uint32_t)std::max(1l, strtol(e, nullptr, 10));
        uint32_t *n_long = arena.alloc_n<uint32_t>(2);
        GN_CUDA(cudaMemsetAsync(n_long, 0, 8, s));
        GN_LAUNCH("k_sw_prepare", n_sel, s,
                  k_sw_prepare<<<blocks_for(n_sel), 256, 0, s>>>(sel, n_sel, (int32_t)p.band_w, qstart_d, B, dp_cells,
                                                                  sw_long, okeys, n_long));
        void *scr = arena.alloc(scan_scratch_bytes(n_sel));
        exclusive_scan_u32(B, soff, n_sel, scr, s);
        uint64_t cells = 0, area[2] = {0, 0};
        GN_CUDA(cudaMemcpyAsync(&cells, soff + n_sel, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        GN_CUDA(cudaMemcpyAsync(area, dp_cells, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        GN_CUDA(cudaStreamSynchronize(s));
        SwCell *strips = arena.alloc_n<SwCell>(cells);
        void *rs = arena.alloc(radix_scratch_bytes(n_sel));
        const uint64_t *order = radix_sort(okeys, okeys_alt, nullptr, nullptr, n_sel, 32, 48, rs, s, TAG_RECORD_SORT)
                                    ? okeys_alt : okeys;
        GN_CUDA(cudaMemsetAsync(counter, 0, 12, s));
        uint32_t *wide = arena.alloc_n<uint32_t>(n_sel);
        // lanes per HSP of the grouped path (the index's tuning; GN_SW_LANES overrides)
        uint32_t sw_lanes = ix->tuning.sw_lanes ? ix->tuning.sw_lanes : 8;
        if (const char *e = getenv("GN_SW_LANES")) sw_lanes = (uint32_t)atoi(e);
        if (sw_lanes != 16 && sw_lanes != 32) sw_lanes = 8;
        auto sw_kernel = sw_lanes == 32 ? k_banded_sw<32, 2> : sw_lanes == 16 ? k_banded_sw<16, 3> : k_banded_sw<8, 5>;
        const uint32_t per_warp = 32 / sw_lanes;
        unsigned warps = (unsigned)std::min<uint64_t>((n_sel + per_warp - 1) / per_warp, (uint64_t)num_sms() * 32);
        GN_LAUNCH("k_banded_sw", area[0], s,
                  sw_kernel<<<(warps * 32 + 127) / 128, 128, 0, s>>>(sel, n_sel, soff, strips, qp.pk, qp.nb, qstart_d,
                                                          ix->bank.pk, ix->bank.nb, ix->seq_start_d, sc.match,
                                                          sc.mismatch, sc.gap_open, sc.gap_extend,
                                                          (int32_t)p.band_w, counter, order, wide, counter + 1,
                                                          n_long, n_long + 1, aln, status));
        GN_LAUNCH("k_banded_sw_wide", area[1], s,
                  k_banded_sw_wide<<<num_sms() * 4, 128, 0, s>>>(sel, wide, counter + 1, counter + 2, soff, strips, qp.pk,
                                                                qp.nb, qstart_d, ix->bank.pk, ix->bank.nb,
                                                                ix->seq_start_d, sc.match, sc.mismatch, sc.gap_open,
                                                                sc.gap_extend, (int32_t)p.band_w, aln, status));
    }
    timer.mark("banded_sw");
    if (keep) {
        std::vector<DevAln> v = to_host(aln, n_sel, s);
        res->st_aln.resize(n_sel);
        for (uint32_t i = 0; i < n_sel; ++i) {
            gn_hit &h = res->st_aln[i];
            h.query = v[i].qi; h.seq = v[i].seq; h.q_start = v[i].qs; h.q_end = v[i].qe;
            h.db_start = v[i].ds; h.db_end = v[i].de; h.score = v[i].score; h.rank = 0; h.evalue = 0; h.bits = 0;
        }
    }

    // a13: duplicates (same query, sequence and ranges: keep the best score), rank by score, statistics
    uint32_t n_out = 0;
    gn_hit *fin = arena.alloc_n<gn_hit>(n_sel);
    const uint64_t *qoff_dev = nullptr;  // per-query offsets of fin, when a phase computed them
    const char *renv = getenv("GN_RANK_PATH");
    const bool per_query_rank = p.max_alignments != 0 && p.max_alignments <= (uint32_t)RQ_CAP &&
                                !(renv && strcmp(renv, "sort") == 0);
    if (n_sel && per_query_rank) {
        uint32_t *qrange = arena.alloc_n<uint32_t>(2ull * nq);
        GN_CUDA(cudaMemsetAsync(qrange, 0, 8ull * nq, s));
        GN_LAUNCH("k_query_ranges", n_sel, s, k_query_ranges<<<blocks_for(n_sel), 256, 0, s>>>(aln, n_sel, qrange));
        gn_hit *hits = arena.alloc_n<gn_hit>(n_sel);
        uint32_t *qcount = arena.alloc_n<uint32_t>(nq);
        const unsigned rgrid = (unsigned)std::min<uint64_t>(nq, (uint64_t)num_sms() * 8);
        GN_LAUNCH("k_rank_query", n_sel, s,
                  k_rank_query<<<rgrid, 256, 0, s>>>(aln, qrange, nq, qstart_d, (double)ix->n_bases, sc.lambda, sc.K,
                                                     p.max_evalue, hits, qcount));
        uint64_t *qoff = arena.alloc_n<uint64_t>(nq + 1);
        void *scr = arena.alloc(scan_scratch_bytes(nq));
        exclusive_scan_u32(qcount, qoff, nq, scr, s);
        qoff_dev = qoff;  // the results' per-query offsets
        uint64_t tot = 0;
        GN_CUDA(cudaMemcpyAsync(&tot, qoff + nq, 8, cudaMemcpyDeviceToHost, s));
        GN_CUDA(cudaStreamSynchronize(s));
        n_out = (uint32_t)tot;
        GN_LAUNCH("k_gather_ranked", n_out, s,
                  k_gather_ranked<<<rgrid, 256, 0, s>>>(hits, qrange, qoff, nq, fin));
    } else if (n_sel) {
        const int scb = std::min(31, bits_for(std::max<uint64_t>(65535, max_qlen) * (uint64_t)std::max(1, sc.match)));
        uint32_t *perm = arena.alloc_n<uint32_t>(n_sel);
        sort_records(reinterpret_cast<const uint32_t *>(aln), ALN_WORDS, n_sel,
                     {{A_QI, qib, false}, {A_SEQ, seqb, false}, {A_QS, qposb, false}, {A_QE, qposb, false},
                      {A_DS, posb, false}, {A_DE, posb, false}, {A_SCORE, scb, true}},
                     perm, arena, s);
        DevAln *srt = arena.alloc_n<DevAln>(n_sel);
        gather_records(reinterpret_cast<const uint32_t *>(aln), ALN_WORDS, perm, n_sel, reinterpret_cast<uint32_t *>(srt), s);
        uint32_t *flag = arena.alloc_n<uint32_t>(n_sel);
        GN_LAUNCH("k_dup_flags", n_sel, s,
                  k_dup_flags<<<blocks_for(n_sel), 256, 0, s>>>(srt, n_sel, flag));
        DevAln *uniq = arena.alloc_n<DevAln>(n_sel);
        uint32_t nu = compact_records(reinterpret_cast<const uint32_t *>(srt), ALN_WORDS, flag, n_sel,
                                      reinterpret_cast<uint32_t *>(uniq), arena, s);
        if (nu) {
            uint32_t *perm2 = arena.alloc_n<uint32_t>(nu);
            sort_records(reinterpret_cast<const uint32_t *>(uniq), ALN_WORDS, nu,
                         {{A_QI, qib, false}, {A_SCORE, scb, true}, {A_SEQ, seqb, false}, {A_QS, qposb, false},
                          {A_DS, posb, false}, {A_QE, qposb, false}, {A_DE, posb, false}},
                         perm2, arena, s);
            DevAln *ranked = arena.alloc_n<DevAln>(nu);
            gather_records(reinterpret_cast<const uint32_t *>(uniq), ALN_WORDS, perm2, nu,
                           reinterpret_cast<uint32_t *>(ranked), s);
            GN_LAUNCH("k_first_of_query", 0, s,
                      k_first_of_query<<<blocks_for(nu), 256, 0, s>>>(reinterpret_cast<const uint32_t *>(ranked), ALN_WORDS, nu, first));
            gn_hit *hits = arena.alloc_n<gn_hit>(nu);
            uint32_t *f2 = arena.alloc_n<uint32_t>(nu);
            GN_LAUNCH("k_finalize", nu, s,
                      k_finalize<<<blocks_for(nu), 256, 0, s>>>(ranked, nu, first, qstart_d, (double)ix->n_bases, sc.lambda, sc.K,
                                                      p.max_evalue, hits, f2));
            static_assert(sizeof(gn_hit) % 4 == 0, "gn_hit words");
            n_out = compact_records(reinterpret_cast<const uint32_t *>(hits), (int)(sizeof(gn_hit) / 4), f2, nu,
                                    reinterpret_cast<uint32_t *>(fin), arena, s);
        }
    }
    timer.mark("rank");
    uint32_t st = 0, wst = 0;
    GN_CUDA(cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaMemcpyAsync(&wst, wait_status, 4, cudaMemcpyDeviceToHost, s));
    res->hits = to_host(fin, n_out, s);
    GN_REQUIRE((wst & DEV_ERR_TIMEOUT) == 0, GN_ETIMEOUT, "a device-side wait ran out (scan look-back)");
#ifdef GN_CHECKS
    uint32_t cbits = 0;
    GN_CUDA(cudaMemcpyAsync(&cbits, check_bits, 4, cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    GN_REQUIRE((cbits & DEV_ERR_BOUNDS) == 0, GN_EINTERNAL, "a device-side bounds check failed (checked build)");
#endif
    GN_REQUIRE((st & DEV_ERR_BOUNDS) == 0, GN_EINTERNAL, "a device-side bounds check failed");
    GN_REQUIRE((st & DEV_ERR_BAND_TOO_WIDE) == 0, GN_ETOOBIG,
               "an alignment band exceeded 65,535 diagonals or its window 2^32 cells");
    if (qoff_dev) {
        res->qoff = to_host(qoff_dev, nq + 1, s);
    } else {
        res->qoff.assign(nq + 1, 0);
        for (uint32_t i = 0; i < n_out; ++i) res->qoff[res->hits[i].query + 1]++;
        for (uint32_t i = 0; i < nq; ++i) res->qoff[i + 1] += res->qoff[i];
    }
    timer.mark("output");
    GN_CUDA(cudaStreamSynchronize(s));
    {
        std::lock_guard<std::mutex> lk(ix->phase_mu);
        timer.finish(ix->last_phases);
        ix->last_kernels.clear();
        for (auto &r : ktimer.recs) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, r.a, r.b);
            auto it = std::find_if(ix->last_kernels.begin(), ix->last_kernels.end(),
                                   [&](const gn_index::KernelStat &k) { return strcmp(k.name, r.name) == 0; });
            if (it == ix->last_kernels.end()) {
                ix->last_kernels.push_back({r.name, 0.0, 0u, 0ull});
                it = ix->last_kernels.end() - 1;
            }
            it->ms += ms;
            it->launches += 1;
            it->units += r.units;
        }
    }

    arena.release();
}

}  // namespace gn
