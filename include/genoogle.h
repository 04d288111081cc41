/*
 * genoogle.h - C ABI of the GB300 (sm_103a) implementation of the Genoogle
 * search path: indexed search of DNA queries against a sequence bank
 * (F. F. Albrecht, "Genoogle: an indexed and parallelized search engine for
 * similar DNA sequences", arXiv 1507.02987).
 *
 * Conventions
 *  - All functions return gn_status; GN_OK is 0.  On failure gn_last_error()
 *    returns a message for the calling thread (valid until its next call).
 *  - Handles (gn_index, gn_results, gn_server) are opaque and owned by the
 *    library; free them with the matching gn_*_free / gn_serve_stop.
 *  - Inputs are copied (host inputs) or only read (device inputs) during the
 *    call; the caller keeps ownership of every pointer it passes.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work of a call is ordered on that stream; the call returns after the
 *    stream has finished the call's work unless stated otherwise.
 *  - Positions are 0-based; ranges are half-open [start, end).
 *  - Bases are ASCII.  A, C, G, T (and U, read as T) in either case are bases;
 *    anything else (N, IUPAC codes) is a non-base: windows holding one are
 *    neither indexed nor looked up, and it scores as a mismatch against
 *    everything in extension and alignment.
 *  - Limits: bank < 2^32 bases in total; query length < 2^24 bases for gn_search
 *    (over 65,535 in overlapping segments) and < 65,536 for the request loop; at
 *    most 65,536 queries (or query segments) per gn_search call; k in 1..16;
 *    stride >= 1.
 */
#ifndef GENOOGLE_H
#define GENOOGLE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GN_API __attribute__((visibility("default")))
#else
#define GN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GN_OK = 0,
    GN_EINVAL = 1,    /* invalid argument (k, stride, lengths, null pointers, ...) */
    GN_ENOMEM = 2,    /* device or host allocation failed */
    GN_ECUDA = 3,     /* a CUDA call or a kernel-side check failed */
    GN_ETIMEOUT = 4,  /* a bounded wait ran out (serving poll, device-side waits of a scan) */
    GN_EBUSY = 5,     /* the server is stopping or its queue is full */
    GN_ETOOBIG = 6,   /* the request exceeds a documented limit or the memory budget */
    GN_EINTERNAL = 7  /* broken internal invariant (a bug) */
} gn_status;

typedef enum { GN_MEM_HOST = 0, GN_MEM_DEVICE = 1 } gn_memory;

/* A sequence bank: sequence s is bases[seq_start[s] .. seq_start[s+1]).
 * seq_start (n_seqs + 1 entries, non-decreasing) is always host memory;
 * bases lives where bases_mem says. */
typedef struct {
    uint32_t n_seqs;
    const uint64_t *seq_start;
    const char *bases;
    gn_memory bases_mem;
} gn_bank;

/* Queries back to back: query i is bases[start[i] .. start[i+1]).  start is host
 * memory; bases lives where bases_mem says. */
typedef struct {
    uint32_t n;
    const uint64_t *start;
    const char *bases;
    gn_memory bases_mem;
} gn_queries;

/* Scores (the paper states none; defaults +1, -3, -5, -2).  A gap of length g
 * scores gap_open + g * gap_extend.  lambda and K are the Karlin-Altschul
 * parameters used for the e-value and the bit ("normalized") score. */
typedef struct {
    int32_t match, mismatch, gap_open, gap_extend;
    double lambda, K;
} gn_scoring;

/* Run-time parameters ("Methods" section: maximum distance between index
 * entries of one HSP, minimum HSP length, drop-off of the extension; "Searching
 * process": maximum quantity of alignments; band of the modified
 * Smith-Waterman). */
typedef struct {
    uint32_t max_hit_distance; /* D: largest query-offset gap between hits of one HSP; 0 = 3 * stride */
    uint32_t min_hsp_len;      /* HSPs shorter than this are dropped; 0 = 2 * k */
    int32_t xdrop;             /* extension stops once the score is more than xdrop below its best */
    uint32_t max_alignments;   /* per query, longest HSPs first; 0 = all */
    uint32_t band_w;           /* band half-width w of the alignment */
    double max_evalue;         /* report alignments with e-value <= this (INFINITY = all) */
    uint32_t flags;            /* GN_FLAG_* */
} gn_params;

#define GN_FLAG_KEEP_STAGES 1u  /* keep every phase's output in the results (tests, debugging) */
#define GN_FLAG_KEEP_HITS 2u    /* also keep the sorted hit list (small inputs only) */
#define GN_FLAG_TIME_KERNELS 4u /* bracket every kernel launch with CUDA events (gn_last_kernel_times) */
/* Both strands (the paper searches the query as given; BLAST-style tools also search
 * its reverse complement): query i of the call is searched as result query 2i (as
 * given) and result query 2i + 1, its reverse complement (A <-> T, C <-> G, U -> A,
 * other bytes unchanged).  Ranges of query 2i + 1 are on the reverse complement;
 * its e-values use the same query length.  At most 32,768 queries per call. */
#define GN_FLAG_BOTH_STRANDS 8u

/* One reported alignment. */
typedef struct {
    uint32_t query;     /* index of the query in the call */
    uint32_t seq;       /* bank sequence id */
    uint32_t q_start, q_end;
    uint32_t db_start, db_end;
    int32_t score;
    uint32_t rank;      /* 0 = best alignment of this query */
    double evalue;
    double bits;
} gn_hit;

/* An HSP (stage outputs): query and bank ranges, length = min of the two spans. */
typedef struct {
    uint32_t query, seq, q_start, q_end, db_start, db_end, len;
} gn_hsp;

typedef struct gn_index gn_index;
typedef struct gn_results gn_results;
typedef struct gn_server gn_server;

/* Defaults: scoring +1/-3/-5/-2 with lambda = 1.3740631, K = 0.711; params
 * D = 0 (3 * stride), min_hsp_len = 0 (2k), xdrop = 20, max_alignments = 100,
 * band_w = 16, max_evalue = INFINITY, flags = 0.  Either pointer may be NULL. */
GN_API gn_status gn_default_params(gn_scoring *scoring, gn_params *params);

/* Builds the inverted index on the device ("Inverted Indexes" section):
 * 2-bit packing of the bank, non-overlapping windows at offsets 0, stride,
 * 2*stride, ... of every sequence (a partial tail is dropped; windows never
 * cross sequences), a histogram over the 4^k buckets, an exclusive scan of it
 * and a stable scatter that keeps each bucket's occurrences in ascending
 * (sequence, position) order.  The packed bank and the index stay resident in
 * device memory until gn_index_free.  k in 1..16, stride >= 1.
 * Errors: GN_EINVAL (bad k/stride/bank), GN_ETOOBIG (bank >= 2^32 bases),
 * GN_ENOMEM, GN_ECUDA. */
GN_API gn_status gn_index_build(const gn_bank *db, int k, int stride, void *cuda_stream, gn_index **out);
GN_API void gn_index_free(gn_index *index);

typedef struct {
    int32_t k, stride;
    uint32_t n_seqs;
    uint64_t n_bases;
    uint64_t n_postings;
    uint64_t device_bytes; /* device memory held by the index (packed bank + index) */
} gn_index_info;
GN_API gn_status gn_index_get_info(const gn_index *index, gn_index_info *info);

/* Execution settings that never change results (0 = the library's default): the
 * fill kernel's tile size in hits (default 50,000) and threads per tile (512 or
 * 256), the raw hits planned per hit bucket (default 4,096 with the repeat
 * filter), the lanes that align one HSP in the alignment kernel's grouped path
 * (8, 16 or 32: four, two or one HSP per warp, for bands of up to 40, 48 or 64
 * diagonals; default 8) and the DP-window rows from which an alignment goes to the
 * anti-diagonal wavefront path (default 512).  They belong to an index (they depend
 * on its occurrence lists). */
typedef struct {
    uint32_t tile_hits;
    uint32_t fill_threads;
    uint32_t bucket_target;
    uint32_t sw_lanes;
    uint32_t sw_wave_rows;
    uint32_t reserved;
} gn_tuning;
GN_API gn_status gn_index_set_tuning(gn_index *index, const gn_tuning *tuning);
GN_API gn_status gn_index_get_tuning(const gn_index *index, gn_tuning *tuning);

/* Autotuner (no counterpart in the paper; it picks what the paper leaves open on a
 * calibration sample of queries, before a run).  With GN_TUNE_BAND it sets
 * params->band_w to the smallest w of 16, 32, 64, 128 for which a band of 2w
 * raises the sample's total alignment score by at most 0.5 % (128 if none does):
 * wider bands recover alignments whose indels drift off the seed diagonal, at a
 * cost that grows with the band.  w changes results, so the caller passes the
 * chosen params to every later search (and to any reference it compares with).  With GN_TUNE_KERNELS it times
 * the search of the sample with several gn_tuning candidates, one group of settings
 * after the other (fill threads and tile size; raw hits per bucket; lanes per HSP
 * and wavefront rows of the alignment kernel), and installs the fastest on the
 * index (and copies it to *tuning if not NULL).  Not to be run
 * concurrently with other searches on the same index.  Errors as gn_search. */
#define GN_TUNE_BAND 1u
#define GN_TUNE_KERNELS 2u
GN_API gn_status gn_autotune(gn_index *index, const gn_queries *sample, const gn_scoring *scoring, gn_params *params,
                             uint32_t what, void *cuda_stream, gn_tuning *tuning);

/* Builds an index of spaced seeds ("Methods": masks after PatternHunter).  mask
 * is a NUL-terminated string of '1' (base kept) and '0' (base removed), 1..32
 * characters with 1..16 ones, e.g. the paper's "111010010100110111".  The bank is
 * cut into windows of strlen(mask) bases at offsets 0, stride, 2 stride, ...; a
 * window is indexed under the code of its kept bases (k = number of ones) unless a
 * kept base is a non-base.  Queries are coded the same way at every offset, and an
 * HSP ends strlen(mask) bases after its last seed.  A mask of k ones is the plain
 * k-mer index.  Errors as gn_index_build, GN_EINVAL for a malformed mask. */
GN_API gn_status gn_index_build_masked(const gn_bank *bank, const char *mask, int stride, void *cuda_stream,
                                       gn_index **out);

/* Index persistence (the paper keeps its index on disk and loads it at start-up,
 * "Inverted Indexes" section).  gn_index_save writes the whole device-resident
 * index (sequence starts, packed bank, bucket starts, occurrences, sequence lookup
 * table) to a file; gn_index_load reads such a file onto the current device and
 * returns a new index owned by the caller (gn_index_free) that searches exactly like
 * the saved one.  Both stage the data through a 64 MiB host buffer.  Errors:
 * GN_EINVAL (file cannot be opened, written or read, not an index file, another
 * format version, inconsistent sizes), GN_ENOMEM, GN_ECUDA. */
GN_API gn_status gn_index_save(const gn_index *index, const char *path);
GN_API gn_status gn_index_load(const char *path, gn_index **out);

/* Copies the index to host memory: bucket_start (4^k + 1 entries) and, for each
 * occurrence, its sequence id and position (n_postings entries each).  Any
 * pointer may be NULL to skip it.  Intended for tests. */
GN_API gn_status gn_index_export(const gn_index *index, uint64_t *bucket_start, uint32_t *post_seq, uint32_t *post_pos);

/* Searches every query against the index ("Searching process", seven phases):
 * rolling k-mer codes of every query offset; lookup of each code's
 * occurrences (hits); grouping of the hits by (query, diagonal) in per-query
 * diagonal buckets (a repeat filter first drops hits alone on their diagonal;
 * overflowing buckets go through a radix sort) and merging of hits at most D
 * query offsets apart on one (sequence, diagonal) into HSPs of length >=
 * min_hsp_len; X-drop ungapped extension of both HSP ends; merging of
 * overlapped HSPs; selection of the longest max_alignments HSPs per query;
 * banded affine-gap Smith-Waterman of each selected HSP; ranking by score with
 * e-value and bit score.  Queries are independent: results do not depend on
 * how queries are grouped into calls.  Results are host memory owned by the
 * library (gn_results_free).
 *
 * Queries of up to 2^24 - 1 bases are taken (the paper's query sets reach 1 Mbp).
 * The seed phases handle at most 65,535 bases at a time: a longer query is cut
 * into segments of 65,535 bases that overlap by 8,192, and the chains found in
 * the segments are joined before extension, which gives exactly the result on
 * the whole query.  Such calls need max_hit_distance + seed span <= 8,192, no
 * GN_FLAG_KEEP_STAGES / GN_FLAG_KEEP_HITS, at most 65,536 segments in all, and
 * bank sequences shorter than 2^32 - 2^24 bases (GN_EINVAL / GN_ETOOBIG
 * otherwise).  The request loop (gn_serve_submit) takes queries of one segment.
 *
 * Errors: GN_EINVAL, GN_ETOOBIG (a query of 2^24 bases or more, more than 65,536
 * queries, an alignment band over 65,535 diagonals or a DP window of 2^32 cells),
 * GN_ENOMEM, GN_ECUDA. */
GN_API gn_status gn_search(const gn_index *index, const gn_queries *queries, const gn_scoring *scoring,
                    const gn_params *params, void *cuda_stream, gn_results **out);
GN_API void gn_results_free(gn_results *results);

/* Ranked alignments of one query ("Searching process", last phase: the alignments
 * sorted by score with e-value and normalized score), in rank order.  *hits stays
 * valid until gn_results_free.  Errors: GN_EINVAL (missing pointer, query index out
 * of range). */
GN_API gn_status gn_results_get(const gn_results *results, uint32_t query, const gn_hit **hits, uint32_t *n);
GN_API gn_status gn_results_count(const gn_results *results, uint32_t *n_queries, uint64_t *n_hits);

/* Phase outputs kept with GN_FLAG_KEEP_STAGES (GN_EINVAL otherwise).
 * Stage ids: GN_STAGE_HSP (HSPs from merged hits), GN_STAGE_EXT (after
 * extension), GN_STAGE_MERGED (after merging overlapped HSPs),
 * GN_STAGE_SELECTED (after selection) - gn_hsp records of all queries, in no
 * particular order; GN_STAGE_ALIGNED - gn_hit records (score and ranges of each
 * selected HSP's alignment, rank and e-value unset); GN_STAGE_HITS (with
 * GN_FLAG_KEEP_HITS) - uint32 quadruples (query, query offset, sequence id,
 * position) of every hit, in no particular order; GN_STAGE_HIT_COUNTS - uint64
 * hit count per query. */
typedef enum {
    GN_STAGE_HSP = 0, GN_STAGE_EXT = 1, GN_STAGE_MERGED = 2, GN_STAGE_SELECTED = 3,
    GN_STAGE_ALIGNED = 4, GN_STAGE_HITS = 5, GN_STAGE_HIT_COUNTS = 6
} gn_stage;
GN_API gn_status gn_results_stage(const gn_results *results, gn_stage stage, const void **data, uint64_t *n);

/* Per-phase device time of the last gn_search on this index handle, in
 * milliseconds (CUDA events); names[i] is a static string.  Returns the
 * number of phases written (<= cap). */
GN_API int gn_last_phase_times(const gn_index *index, const char **names, float *ms, int cap);

/* Per-kernel device time of the last gn_search on this index handle that ran
 * with GN_FLAG_TIME_KERNELS: for each kernel name, the summed duration of its
 * launches (CUDA events on the launching stream), the number of launches and
 * the summed work items (keys, hits, HSPs or DP cells, per kernel).  Returns
 * the number of kernels written (<= cap). */
GN_API int gn_last_kernel_times(const gn_index *index, const char **names, double *ms, uint32_t *launches,
                                uint64_t *units, int cap);

/* Number of kernels this library has launched in the process so far. */
GN_API uint64_t gn_kernel_launch_count(void);

/* ----------------------------------------------------------- serving ---
 * Request loop with continuous batching (the paper's web-services interface,
 * "Implementation" section, as a resident-index service).  Three worker
 * threads, each with its own CUDA stream, take submitted queries in arrival
 * order while their footprint fits mem_budget, run them as one micro-batch
 * (a gn_search on that worker's stream) while other micro-batches still run,
 * and make each result available to gn_serve_poll / gn_serve_poll_any.
 * A query's footprint is its exact seed-hit count times 24 bytes, plus 64
 * bytes per base, 16 KiB of hit buckets and the records of its selected HSPs;
 * each micro-batch also counts 16 MiB of fixed device memory.  The workers
 * count the hits of waiting queries on the device, in arrival order and many at
 * a time, before admitting them; when nothing runs, the oldest query starts at
 * once, alone, with the whole budget (its hit storage capped to what the budget
 * leaves), without waiting for its count.  Each query's result is identical to a gn_search of that
 * query alone.  mem_budget must exceed 16 MiB (GN_EINVAL otherwise).  The server
 * searches queries as given (GN_FLAG_BOTH_STRANDS and GN_FLAG_KEEP_* are ignored). */
GN_API gn_status gn_serve_start(const gn_index *index, const gn_scoring *scoring, const gn_params *params,
                         uint64_t mem_budget, gn_server **out);
/* Thread-safe; copies the query and queues it (no other work on the caller's thread).
 * GN_ETOOBIG for a query of 65,536 bases or more; a query whose footprint alone exceeds
 * the budget fails later, at poll, with GN_ETOOBIG. */
GN_API gn_status gn_serve_submit(gn_server *server, const char *bases, uint32_t len, uint64_t *ticket);
/* Waits up to timeout_ms for the given ticket; GN_ETIMEOUT if not done yet.  On
 * GN_OK *out holds a one-query result owned by the caller (gn_results_free).  A
 * ticket that failed returns its error: GN_ETOOBIG (the query alone exceeds the
 * budget), or the error of its micro-batch (GN_ENOMEM, GN_ECUDA, ...) for each of
 * the batch's tickets; the server keeps serving. */
GN_API gn_status gn_serve_poll(gn_server *server, uint64_t ticket, uint32_t timeout_ms, gn_results **out);
/* Completion queue: waits up to timeout_ms for any finished ticket and returns
 * the oldest one in *ticket (GN_ETIMEOUT and *ticket = 0 if none finished).  On
 * GN_OK *out holds its one-query result; any other status is that ticket's error
 * (as gn_serve_poll). */
GN_API gn_status gn_serve_poll_any(gn_server *server, uint32_t timeout_ms, uint64_t *ticket, gn_results **out);
/* Counters of a server since its start (for monitoring and tests). */
typedef struct {
    uint64_t requests;        /* queries admitted to micro-batches */
    uint64_t batches;         /* micro-batches launched */
    uint64_t max_batch;       /* most queries in one micro-batch */
    uint64_t max_concurrent;  /* most micro-batches in flight at once */
    uint64_t peak_in_use;     /* most budget bytes admitted at once */
    uint64_t in_use;          /* budget bytes admitted now */
    uint64_t queued;          /* submitted queries not admitted yet */
} gn_serve_stats;
GN_API gn_status gn_serve_get_stats(gn_server *server, gn_serve_stats *out);
/* Finishes admitted work, rejects new submissions, joins the server thread, frees the server. */
GN_API gn_status gn_serve_stop(gn_server *server);

/* ------------------------------------------- allocation-free alignment ---
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory on their path - code whose device memory is
 * owned by another allocator that must stay the only one, code running near a
 * hard memory limit that cannot risk an allocation failure mid-job, or loops
 * that cannot afford an allocation call.  It aligns caller-given HSPs exactly
 * as the alignment phase of gn_search does (same band, recurrence, tie-breaks
 * and output as its GN_STAGE_ALIGNED records: query, seq, ranges and score;
 * rank, evalue and bits are 0) and allocates nothing: its scratch (one row
 * strip per warp for 512 warps, bands of at most 1,024 diagonals; about 8 MiB)
 * is a static array in the library's device image, which every GPU that loads
 * the library holds until the process exits.
 *   query_bases  device memory, ASCII, queries back to back
 *   query_start  device memory, n_queries + 1 offsets into query_bases
 *   hsps, out    device memory, n_hsps records each (caller-owned); out[i]
 *                is the alignment of hsps[i]; db ranges are positions in
 *                bank sequence hsps[i].seq of the index
 *   band_w       band half-width w (2*w + 1 <= 1024)
 * The first call on a device looks up the scratch array's address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array and clears its counters first:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * not be issued.  The call returns after the stream has finished.  Errors:
 * GN_ETOOBIG if band_w is too large or an HSP's band spans more than 1,024
 * diagonals (that HSP's record is written with score 0), GN_EINVAL for a
 * missing pointer or an HSP naming a query or sequence that does not exist. */
GN_API gn_status gn_align_hsps_static(const gn_index *index, const char *query_bases, const uint64_t *query_start,
                                      uint32_t n_queries, const gn_hsp *hsps, uint32_t n_hsps,
                                      const gn_scoring *scoring, uint32_t band_w, gn_hit *out, void *cuda_stream);

/* ------------------------------------------------ integer-pipe peaks ---
 * Measured throughput of this GPU's integer pipes (no counterpart in the paper: it
 * is the denominator of the alignment kernel's roofline).  Each figure is operations
 * per second over the whole device, with every SM filled: a three-input add (2
 * operations), max(a + b, c) as plain C (2), the DPX add-max __viaddmax_s32 (2 in
 * one instruction), the DPX three-way max __vimax3_s32 (2), and the DPX max with its
 * predicate __vibmax_s32 after an add (2, plus a select by the predicate).  Runs for
 * some milliseconds on cuda_stream and allocates 64 bytes of device memory.
 * Errors: GN_EINVAL (out is NULL), GN_ENOMEM, GN_ECUDA. */
typedef struct {
    double add3_ops, addmax_plain_ops, dpx_addmax_ops, dpx_max3_ops, dpx_bmax_ops;
    uint32_t sms;
} gn_int_peaks;
GN_API gn_status gn_measure_int_peaks(gn_int_peaks *out, void *cuda_stream);

/* ----------------------------------------------------- fault injection ---
 * For tests of the error paths (the paper has no counterpart).  gn_debug_fail_alloc(n)
 * makes the n-th device allocation that a search (gn_search, or a micro-batch of the
 * request loop) makes from now on fail as if the device were out of memory: the call
 * then returns GN_ENOMEM (a micro-batch fails its tickets with GN_ENOMEM) after freeing
 * what it held.  n = 0 disables it.  gn_debug_alloc_count is the number of such
 * allocations made so far in the process, gn_debug_live_allocs the number held now
 * (0 between calls). */
GN_API void gn_debug_fail_alloc(uint64_t nth);
/* The library's single-pass scan (decoupled look-back: each block of the launch waits for
 * the blocks before it to publish their sums), for tests of its bounded wait:
 * out[i] = in[0] + ... + in[i-1] and out[n] = the total; in (n uint32) and out (n + 1
 * uint64) are device memory.  wait_cycles bounds each block's wait (SM clock cycles;
 * 0 = the library's default, about a second); drop_first = 1 keeps the first tile of
 * 2,048 elements from publishing its sum, so that the waits behind it run out.  Returns
 * GN_ETIMEOUT if a wait ran out (out is then wrong), after the stream has finished. */
GN_API gn_status gn_debug_scan(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t wait_cycles, int drop_first,
                               void *cuda_stream);
/* The library's LSD radix sort, for tests: sorts keys (n uint64, device memory) in place,
 * stably, by bits [bit_lo, bit_hi) (8 bits per pass), with vals (n uint32, device memory,
 * or NULL) moved along.  Sorts of at most 4,096 keys run every pass in one launch of one
 * block; sorts of up to 2^27 keys take the single-pass form (one histogram launch, then
 * one launch per pass whose blocks wait, with decoupled look-back, for the blocks before
 * them to publish their digit counts); three_kernel = 1 forces the three-kernel passes
 * (upsweep, scan, downsweep) that larger sorts take.  wait_cycles and
 * drop_first (the first tile of 4,096 keys publishes nothing) as in gn_debug_scan.
 * Errors: GN_EINVAL (keys NULL with n > 0, bits outside 0 <= bit_lo <= bit_hi <= 64),
 * GN_ETOOBIG (n >= 2^32), GN_ENOMEM, GN_ETIMEOUT if a wait ran out (the keys are then
 * wrong), GN_ECUDA.  Returns after the stream has finished. */
GN_API gn_status gn_debug_sort(uint64_t *keys, uint32_t *vals, uint64_t n, int bit_lo, int bit_hi,
                               uint64_t wait_cycles, int drop_first, int three_kernel, void *cuda_stream);
GN_API uint64_t gn_debug_alloc_count(void);
GN_API int64_t gn_debug_live_allocs(void);

/* Message of the last failing call on this thread ("" if none). */
GN_API const char *gn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GENOOGLE_H */
