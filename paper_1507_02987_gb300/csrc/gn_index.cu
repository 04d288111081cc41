// gn_index.cu - device construction of the inverted index ("Inverted Indexes"
// section of the paper): the bank is packed to 2 bits per base, cut into
// non-overlapping windows at offsets 0, t, 2t, ... of every sequence, and each
// window's occurrence is filed under its k-mer code.  Buckets are a CSR
// structure: off[c] .. off[c+1] index the occurrences of code c, in ascending
// (sequence, position) order, stored as the window's global base offset.
#include <algorithm>

#include <cstdio>
#include <cstring>
#include <string>

#include "gn_internal.cuh"

namespace gn {

// windows per sequence: len >= span ? (len - span) / t + 1 : 0 (span = k without a mask)
__global__ void k_window_counts(const uint64_t *__restrict__ seq_start, uint32_t n_seqs, int span, int t,
                                uint32_t *__restrict__ wcnt) {
    uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seqs) return;
    uint64_t L = seq_start[s + 1] - seq_start[s];
    wcnt[s] = L >= (uint64_t)span ? (uint32_t)((L - span) / t + 1) : 0u;
}

constexpr int WIN_J = 8;  // windows per lane per warp chunk

// Pass 1 (flags = true): validity flag of every window + bucket histogram.
// Pass 2 (flags = false): key (code << 32 | global offset) of every valid window at its compacted slot.
template <bool FLAGS>
__global__ void k_bank_windows(const uint64_t *__restrict__ seq_start, const uint64_t *__restrict__ woff,
                               uint32_t n_seqs, uint64_t W, const uint32_t *__restrict__ pk,
                               const uint32_t *__restrict__ nb, SeedShape sh, int t, uint32_t *__restrict__ flags,
                               uint32_t *__restrict__ hist, const uint64_t *__restrict__ slot,
                               uint64_t *__restrict__ keys) {
    const int lane = threadIdx.x & 31;
    uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t w0 = warp * 32 * WIN_J;
    if (w0 >= W) return;
    uint32_t s = 0;
    if (lane == 0) s = dev_upper_index(woff, n_seqs + 1, w0);
    s = __shfl_sync(0xffffffffu, s, 0);
#pragma unroll
    for (int it = 0; it < WIN_J; ++it) {
        uint64_t w = w0 + (uint64_t)it * 32 + lane;
        if (w >= W) break;
        while (woff[s + 1] <= w) ++s;
        uint64_t g = seq_start[s] + (w - woff[s]) * (uint64_t)t;
        bool bad = dev_seed_has_nonbase(nb, g, sh);
        uint32_t code = dev_seed_code(pk, g, sh);
        if (FLAGS) {
            flags[w] = bad ? 0u : 1u;
            if (!bad) atomicAdd(&hist[code], 1u);
        } else if (!bad) {
            keys[slot[w]] = ((uint64_t)code << 32) | g;
        }
    }
}

__global__ void k_low_words(const uint64_t *__restrict__ keys, uint64_t n, uint32_t *__restrict__ out) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)keys[i];
}

// lut[j] = last sequence s with start[s] <= j << SEQ_LUT_SHIFT (positions past the bank
// map to the last sequence).
__global__ void k_seq_lut(const uint64_t *__restrict__ start, uint32_t ns, uint64_t n, uint64_t nlut,
                          uint32_t *__restrict__ lut) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nlut) return;
    const uint64_t x = min(j << SEQ_LUT_SHIFT, n > 0 ? n - 1 : 0);
    lut[j] = dev_upper_index(start, ns, x);  // over the ns starts: the result is < ns
}

// Seeds of `span` bases keeping the positions set in `keep` (k of them).
static void index_build_shape(const gn_bank *db, int k, int span, uint32_t keep, int t, cudaStream_t s, gn_index *ix);

void index_build(const gn_bank *db, int k, int t, cudaStream_t s, gn_index *ix) {
    GN_REQUIRE(k >= 1 && k <= 16, GN_EINVAL, "k must be in 1..16");
    index_build_shape(db, k, k, (uint32_t)((1ull << k) - 1ull), t, s, ix);
}

// "Methods": a mask such as 111010010100110111 ('1' = base kept, '0' = removed) over
// windows of the mask's length.
void index_build_masked(const gn_bank *db, const char *mask, int t, cudaStream_t s, gn_index *ix) {
    GN_REQUIRE(mask, GN_EINVAL, "mask is required");
    const size_t span = strlen(mask);
    GN_REQUIRE(span >= 1 && span <= 32, GN_EINVAL, "a mask has 1..32 positions");
    uint32_t keep = 0;
    int k = 0;
    for (size_t i = 0; i < span; ++i) {
        GN_REQUIRE(mask[i] == '0' || mask[i] == '1', GN_EINVAL, "a mask holds only '0' and '1'");
        if (mask[i] == '1') { keep |= 1u << i; ++k; }
    }
    GN_REQUIRE(k >= 1 && k <= 16, GN_EINVAL, "a mask keeps 1..16 positions");
    index_build_shape(db, k, (int)span, keep, t, s, ix);
}

static void index_build_shape(const gn_bank *db, int k, int span, uint32_t keep, int t, cudaStream_t s,
                              gn_index *ix) {
    GN_REQUIRE(db && db->seq_start, GN_EINVAL, "bank and bank.seq_start are required");
    GN_REQUIRE(t >= 1, GN_EINVAL, "stride must be >= 1");
    const uint32_t ns = db->n_seqs;
    const uint64_t n = db->seq_start[ns] - db->seq_start[0];
    GN_REQUIRE(db->seq_start[0] == 0, GN_EINVAL, "bank.seq_start[0] must be 0");
    GN_REQUIRE(n < (1ull << 32), GN_ETOOBIG, "bank must hold fewer than 2^32 bases");
    GN_REQUIRE(n == 0 || db->bases, GN_EINVAL, "bank.bases is required");
    uint64_t maxlen = 0;
    for (uint32_t i = 0; i < ns; ++i) {
        GN_REQUIRE(db->seq_start[i + 1] >= db->seq_start[i], GN_EINVAL, "bank.seq_start must be non-decreasing");
        maxlen = std::max<uint64_t>(maxlen, db->seq_start[i + 1] - db->seq_start[i]);
    }
    GN_CUDA(cudaGetDevice(&ix->device));
    configure_mempool(ix->device);
    ix->k = k;
    ix->t = t;
    ix->span = span;
    ix->keep = keep;
    ix->n_seqs = ns;
    ix->n_bases = n;
    ix->max_seq_len = (uint32_t)maxlen;
    ix->seq_start_h.assign(db->seq_start, db->seq_start + ns + 1);
    const SeedShape sh{k, span, keep};

    const uint64_t nbk = 1ull << (2 * k);
    uint64_t bytes = 0;
    GN_CUDA(cudaMalloc(&ix->seq_start_d, sizeof(uint64_t) * (ns + 1)));
    bytes += sizeof(uint64_t) * (ns + 1);
    GN_CUDA(cudaMalloc(&ix->bank.pk, 4 * Packed::pk_words(n)));
    GN_CUDA(cudaMalloc(&ix->bank.nb, 4 * Packed::nb_words(n)));
    bytes += 4 * (Packed::pk_words(n) + Packed::nb_words(n));
    GN_CUDA(cudaMalloc(&ix->off_d, sizeof(uint64_t) * (nbk + 1)));
    bytes += sizeof(uint64_t) * (nbk + 1);
    GN_CUDA(cudaMemcpyAsync(ix->seq_start_d, ix->seq_start_h.data(), sizeof(uint64_t) * (ns + 1),
                            cudaMemcpyHostToDevice, s));
    // sequence lookup table: the sequence holding each block of 2^SEQ_LUT_SHIFT bases
    const uint64_t nlut = (n >> SEQ_LUT_SHIFT) + 1;
    GN_CUDA(cudaMalloc(&ix->seq_lut_d, sizeof(uint32_t) * nlut));
    bytes += sizeof(uint32_t) * nlut;
    if (ns > 0)
        GN_LAUNCH("k_seq_lut", nlut, s,
                  k_seq_lut<<<(unsigned)((nlut + 255) / 256), 256, 0, s>>>(ix->seq_start_d, ns, n, nlut, ix->seq_lut_d));
    else
        GN_CUDA(cudaMemsetAsync(ix->seq_lut_d, 0, sizeof(uint32_t) * nlut, s));

    DeviceArena arena(s);
    uint32_t *wait_status = arena.alloc_n<uint32_t>(1);  // bounded waits of the scans
    GN_CUDA(cudaMemsetAsync(wait_status, 0, 4, s));
    WaitStatusScope wscope(wait_status);
    // K1: 2-bit packing of the bank
    const uint8_t *bases_d = reinterpret_cast<const uint8_t *>(db->bases);
    if (db->bases_mem == GN_MEM_HOST && n > 0) {
        uint8_t *tmp = arena.alloc_n<uint8_t>(n);
        GN_CUDA(cudaMemcpyAsync(tmp, db->bases, n, cudaMemcpyHostToDevice, s));
        bases_d = tmp;
    }
    pack_bases(bases_d, n, ix->bank, s);

    // windows per sequence and their exclusive scan
    uint32_t *wcnt = arena.alloc_n<uint32_t>(ns);
    uint64_t *woff = arena.alloc_n<uint64_t>(ns + 1);
    if (ns) {
        GN_LAUNCH("k_window_counts", ns, s,
                  k_window_counts<<<(ns + 255) / 256, 256, 0, s>>>(ix->seq_start_d, ns, span, t, wcnt));
    }
    void *scan_scr = arena.alloc(std::max(scan_scratch_bytes(ns), scan_scratch_bytes(nbk)));
    exclusive_scan_u32(wcnt, woff, ns, scan_scr, s);
    uint64_t W = 0;
    GN_CUDA(cudaMemcpyAsync(&W, woff + ns, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));

    // K2: window validity + bucket histogram
    uint32_t *hist = arena.alloc_n<uint32_t>(nbk);
    GN_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nbk, s));
    uint32_t *flags = arena.alloc_n<uint32_t>(W);
    uint64_t *slot = arena.alloc_n<uint64_t>(W + 1);
    uint64_t warps = (W + 32 * WIN_J - 1) / (32 * WIN_J);
    unsigned grid = (unsigned)std::max<uint64_t>(1, (warps * 32 + 255) / 256);
    if (W) {
        GN_LAUNCH("k_bank_windows_flags", W, s,
                  k_bank_windows<true><<<grid, 256, 0, s>>>(ix->seq_start_d, woff, ns, W, ix->bank.pk, ix->bank.nb, sh, t,
                                                  flags, hist, nullptr, nullptr));
    }
    // K3: bucket starts = exclusive scan of the histogram
    exclusive_scan_u32(hist, ix->off_d, nbk, scan_scr, s);
    void *scan_scr2 = arena.alloc(scan_scratch_bytes(W));
    exclusive_scan_u32(flags, slot, W, scan_scr2, s);
    uint64_t P = 0;
    GN_CUDA(cudaMemcpyAsync(&P, ix->off_d + nbk, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    ix->n_postings = P;

    // K4: stable scatter = stable radix sort of (code, global offset) keys by code
    uint64_t *keys = arena.alloc_n<uint64_t>(P);
    uint64_t *keys_alt = arena.alloc_n<uint64_t>(P);
    if (W) {
        GN_LAUNCH("k_bank_windows_keys", W, s,
                  k_bank_windows<false><<<grid, 256, 0, s>>>(ix->seq_start_d, woff, ns, W, ix->bank.pk, ix->bank.nb, sh, t,
                                                   nullptr, nullptr, slot, keys));
    }
    void *rs = arena.alloc(radix_scratch_bytes(P));
    bool flipped = radix_sort(keys, keys_alt, nullptr, nullptr, P, 32, 32 + 2 * k, rs, s, TAG_INDEX_SORT);
    GN_CUDA(cudaMalloc(&ix->post_d, sizeof(uint32_t) * post_alloc_entries(P)));
    bytes += sizeof(uint32_t) * P;
    if (P) {
        GN_LAUNCH("k_low_words", P, s,
                  k_low_words<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(flipped ? keys_alt : keys, P, ix->post_d));
    }
    uint32_t wst = 0;
    GN_CUDA(cudaMemcpyAsync(&wst, wait_status, 4, cudaMemcpyDeviceToHost, s));
    arena.release();
    GN_CUDA(cudaStreamSynchronize(s));
    GN_REQUIRE((wst & DEV_ERR_TIMEOUT) == 0, GN_ETIMEOUT, "a device-side wait ran out (scan look-back)");
    ix->device_bytes = bytes;
}

void index_free(gn_index *ix) {
    if (!ix) return;
    cudaFree(ix->seq_start_d);
    cudaFree(ix->seq_lut_d);
    cudaFree(ix->bank.pk);
    cudaFree(ix->bank.nb);
    cudaFree(ix->off_d);
    cudaFree(ix->post_d);
}

void index_export(const gn_index *ix, uint64_t *bucket_start, uint32_t *post_seq, uint32_t *post_pos) {
    const uint64_t nbk = 1ull << (2 * ix->k);
    if (bucket_start) GN_CUDA(cudaMemcpy(bucket_start, ix->off_d, sizeof(uint64_t) * (nbk + 1), cudaMemcpyDeviceToHost));
    if (!post_seq && !post_pos) return;
    std::vector<uint32_t> g(ix->n_postings);
    if (ix->n_postings)
        GN_CUDA(cudaMemcpy(g.data(), ix->post_d, sizeof(uint32_t) * ix->n_postings, cudaMemcpyDeviceToHost));
    // decode global offsets to (sequence, position) for the caller
    const std::vector<uint64_t> &st = ix->seq_start_h;
    for (uint64_t i = 0; i < ix->n_postings; ++i) {
        uint32_t sidx = (uint32_t)(std::upper_bound(st.begin(), st.end(), (uint64_t)g[i]) - st.begin()) - 1;
        if (post_seq) post_seq[i] = sidx;
        if (post_pos) post_pos[i] = (uint32_t)(g[i] - st[sidx]);
    }
}

// --------------------------------------------------------- persistence --
// File layout (little-endian): a header of 16 uint64 (magic, version, k, stride,
// n_seqs, n_bases, n_postings, max_seq_len, word counts of the sections that
// follow, seed span and kept-position mask), then the sections in order: sequence starts (n_seqs + 1 uint64), packed
// bank words, non-base words, bucket starts (4^k + 1 uint64), occurrences
// (n_postings uint32), sequence lookup table.  Device arrays move through a bounded
// host buffer, so an index of any size needs only that much host memory.
constexpr uint64_t IX_MAGIC = 0x31584449474F4E47ull;  // "GNOGIDX1"
constexpr uint64_t IX_VERSION = 2;
constexpr size_t IX_CHUNK = 64ull << 20;

namespace {
struct FileCloser {
    FILE *f;
    ~FileCloser() { if (f) fclose(f); }
};
void write_all(FILE *f, const void *p, size_t bytes) {
    GN_REQUIRE(bytes == 0 || fwrite(p, 1, bytes, f) == bytes, GN_EINVAL, "index file: write failed");
}
void read_all(FILE *f, void *p, size_t bytes) {
    GN_REQUIRE(bytes == 0 || fread(p, 1, bytes, f) == bytes, GN_EINVAL, "index file: truncated or unreadable");
}
void write_device(FILE *f, const void *d, size_t bytes, std::vector<uint8_t> &buf) {
    for (size_t o = 0; o < bytes; o += IX_CHUNK) {
        const size_t n = std::min(IX_CHUNK, bytes - o);
        GN_CUDA(cudaMemcpy(buf.data(), static_cast<const uint8_t *>(d) + o, n, cudaMemcpyDeviceToHost));
        write_all(f, buf.data(), n);
    }
}
void read_device(FILE *f, void *d, size_t bytes, std::vector<uint8_t> &buf) {
    for (size_t o = 0; o < bytes; o += IX_CHUNK) {
        const size_t n = std::min(IX_CHUNK, bytes - o);
        read_all(f, buf.data(), n);
        GN_CUDA(cudaMemcpy(static_cast<uint8_t *>(d) + o, buf.data(), n, cudaMemcpyHostToDevice));
    }
}
}  // namespace

void index_save(const gn_index *ix, const char *path) {
    GN_REQUIRE(path, GN_EINVAL, "path is required");
    FILE *f = fopen(path, "wb");
    GN_REQUIRE(f, GN_EINVAL, std::string("cannot create ") + path);
    FileCloser fc{f};
    GN_CUDA(cudaSetDevice(ix->device));
    const uint64_t npk = Packed::pk_words(ix->n_bases), nnb = Packed::nb_words(ix->n_bases);
    const uint64_t nbk = (1ull << (2 * ix->k)) + 1, nlut = (ix->n_bases >> SEQ_LUT_SHIFT) + 1;
    uint64_t hdr[16] = {IX_MAGIC, IX_VERSION, (uint64_t)ix->k, (uint64_t)ix->t, ix->n_seqs, ix->n_bases,
                        ix->n_postings, ix->max_seq_len, npk, nnb, nbk, nlut, (uint64_t)ix->span, ix->keep, 0, 0};
    write_all(f, hdr, sizeof(hdr));
    write_all(f, ix->seq_start_h.data(), sizeof(uint64_t) * (ix->n_seqs + 1));
    std::vector<uint8_t> buf(IX_CHUNK);
    write_device(f, ix->bank.pk, 4 * npk, buf);
    write_device(f, ix->bank.nb, 4 * nnb, buf);
    write_device(f, ix->off_d, 8 * nbk, buf);
    write_device(f, ix->post_d, 4 * ix->n_postings, buf);
    write_device(f, ix->seq_lut_d, 4 * nlut, buf);
    GN_REQUIRE(fflush(f) == 0, GN_EINVAL, "index file: write failed");
}

void index_load(const char *path, gn_index *ix) {
    GN_REQUIRE(path, GN_EINVAL, "path is required");
    FILE *f = fopen(path, "rb");
    GN_REQUIRE(f, GN_EINVAL, std::string("cannot open ") + path);
    FileCloser fc{f};
    uint64_t hdr[16];
    read_all(f, hdr, sizeof(hdr));
    GN_REQUIRE(hdr[0] == IX_MAGIC, GN_EINVAL, "not an index file");
    GN_REQUIRE(hdr[1] == IX_VERSION, GN_EINVAL, "unsupported index file version");
    const int k = (int)hdr[2], t = (int)hdr[3];
    GN_REQUIRE(k >= 1 && k <= 16 && t >= 1, GN_EINVAL, "index file: bad k or stride");
    const uint64_t ns = hdr[4], n = hdr[5], np = hdr[6];
    GN_REQUIRE(ns < (1ull << 32) && n < (1ull << 32) && np <= n, GN_EINVAL, "index file: bad sizes");
    const uint64_t npk = Packed::pk_words(n), nnb = Packed::nb_words(n);
    const uint64_t nbk = (1ull << (2 * k)) + 1, nlut = (n >> SEQ_LUT_SHIFT) + 1;
    GN_REQUIRE(hdr[8] == npk && hdr[9] == nnb && hdr[10] == nbk && hdr[11] == nlut, GN_EINVAL,
               "index file: section sizes do not match the header");
    GN_CUDA(cudaGetDevice(&ix->device));
    configure_mempool(ix->device);
    ix->k = k;
    ix->t = t;
    ix->span = (int)hdr[12];
    ix->keep = (uint32_t)hdr[13];
    GN_REQUIRE(ix->span >= k && ix->span <= 32 && __builtin_popcount(ix->keep) == k &&
                   (ix->span == 32 || (ix->keep >> ix->span) == 0),
               GN_EINVAL, "index file: bad seed shape");
    ix->n_seqs = (uint32_t)ns;
    ix->n_bases = n;
    ix->n_postings = np;
    ix->max_seq_len = (uint32_t)hdr[7];
    ix->seq_start_h.resize(ns + 1);
    read_all(f, ix->seq_start_h.data(), sizeof(uint64_t) * (ns + 1));
    GN_REQUIRE(ix->seq_start_h[0] == 0 && ix->seq_start_h[ns] == n, GN_EINVAL, "index file: bad sequence starts");
    for (uint64_t i = 0; i < ns; ++i)
        GN_REQUIRE(ix->seq_start_h[i + 1] >= ix->seq_start_h[i], GN_EINVAL, "index file: bad sequence starts");
    uint64_t bytes = 0;
    GN_CUDA(cudaMalloc(&ix->seq_start_d, sizeof(uint64_t) * (ns + 1)));
    GN_CUDA(cudaMalloc(&ix->bank.pk, 4 * npk));
    GN_CUDA(cudaMalloc(&ix->bank.nb, 4 * nnb));
    GN_CUDA(cudaMalloc(&ix->off_d, 8 * nbk));
    GN_CUDA(cudaMalloc(&ix->post_d, 4 * post_alloc_entries(np)));
    GN_CUDA(cudaMalloc(&ix->seq_lut_d, 4 * nlut));
    ix->bank.n = n;
    bytes += 8 * (ns + 1) + 4 * (npk + nnb) + 8 * nbk + 4 * np + 4 * nlut;
    GN_CUDA(cudaMemcpy(ix->seq_start_d, ix->seq_start_h.data(), 8 * (ns + 1), cudaMemcpyHostToDevice));
    std::vector<uint8_t> buf(IX_CHUNK);
    read_device(f, ix->bank.pk, 4 * npk, buf);
    read_device(f, ix->bank.nb, 4 * nnb, buf);
    read_device(f, ix->off_d, 8 * nbk, buf);
    read_device(f, ix->post_d, 4 * np, buf);
    read_device(f, ix->seq_lut_d, 4 * nlut, buf);
    uint64_t last = 0;
    GN_CUDA(cudaMemcpy(&last, ix->off_d + (nbk - 1), 8, cudaMemcpyDeviceToHost));
    GN_REQUIRE(last == np, GN_EINVAL, "index file: bucket starts do not end at the occurrence count");
    ix->device_bytes = bytes;
}

}  // namespace gn
