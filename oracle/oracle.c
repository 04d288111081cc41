/*
 * oracle.c - plain, slow, obviously correct CPU implementation of the Genoogle
 * search path (arXiv 1507.02987).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the CUDA
 * implementation.
 *
 * Every step follows the paper's text (section names below) with the readings
 * listed in the design notes of the repository:
 *   encoding            - "Methods": 2 bits per base, sub-sequences of 1..16 bases
 *   bank windows        - "Methods": non-overlapping windows for the bank
 *   inverted index      - "Inverted Indexes": 4^k buckets, each occurrence is a
 *                         (sequence id, position) pair of two 4-byte integers,
 *                         built with the sort-based inversion (here a counting sort,
 *                         which is the same stable ordering by (code, seq, pos))
 *   search phases       - "Searching process", the seven phases in order
 *   statistics          - Karlin-Altschul E-value and bit score (the paper reports
 *                         "e-value, score, normalized score" without a formula)
 *
 * Data structures are the plainest ones: arrays, qsort, a full band DP.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NEG (-(1 << 29)) /* "minus infinity" for gap states; far from overflow */

/* ------------------------------------------------------------ encoding --- */
/* "Methods": A, C, G, T (U for RNA) coded in 2 bits; first base of a
 * sub-sequence in the most significant bits.  Anything else is not a base. */
static int base_code(uint8_t b) {
    switch (b) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': case 'U': case 'u': return 3;
    default: return -1;
    }
}

/* "Methods" (masks): a seed is `span` consecutive bases of which the mask keeps
 * some (mask[i] == '1'); its code is the kept bases in order, first one most
 * significant.  -1 if a kept base is not a base.  A plain k-base window is the
 * mask of k ones. */
static int64_t seed_code(const uint8_t *s, const char *mask, int span) {
    int64_t code = 0;
    for (int i = 0; i < span; ++i) {
        if (mask[i] != '1') continue;
        int c = base_code(s[i]);
        if (c < 0) return -1;
        code = code * 4 + c;
    }
    return code;
}

/* ------------------------------------------------------- inverted index --- */
typedef struct {
    int32_t k, t;                /* k: kept bases of a seed (its code has 2k bits) */
    int32_t span;                /* bases a seed covers (the mask length; k without a mask) */
    char mask[33];               /* '1' = kept, '0' = removed */
    uint32_t n_seqs;
    const uint64_t *seq_start;   /* borrowed, n_seqs + 1 */
    const uint8_t *bases;        /* borrowed */
    uint64_t n_buckets;          /* 4^k */
    uint64_t *bucket_start;      /* n_buckets + 1 */
    uint32_t *post_seq;          /* sequence id of each occurrence */
    uint32_t *post_pos;          /* position inside the sequence */
    uint64_t n_postings;
} or_index;

/* "Inverted Indexes": one bucket per possible sub-sequence; the bank is cut into
 * non-overlapping windows at offsets 0, t, 2t, ... of every sequence (a partial
 * tail is dropped, windows never cross sequences, windows holding a non-base at a
 * kept position are not indexed).  With a mask ("Methods"; the paper's example
 * keeps 11 of 18 bases) a window covers the mask's length and is indexed under the
 * code of its kept bases.  Occurrences in a bucket are in ascending (sequence,
 * position). */
or_index *or_index_build_masked(const uint8_t *bases, const uint64_t *seq_start, uint32_t n_seqs, const char *mask,
                                int t) {
    int span = (int)strlen(mask), k = 0;
    if (span < 1 || span > 32 || t < 1) return NULL;
    for (int i = 0; i < span; ++i) {
        if (mask[i] == '1') ++k;
        else if (mask[i] != '0') return NULL;
    }
    if (k < 1 || k > 16) return NULL;
    or_index *ix = (or_index *)calloc(1, sizeof(or_index));
    ix->k = k; ix->t = t; ix->span = span; ix->n_seqs = n_seqs; ix->seq_start = seq_start; ix->bases = bases;
    memcpy(ix->mask, mask, (size_t)span + 1);
    ix->n_buckets = (uint64_t)1 << (2 * k);
    ix->bucket_start = (uint64_t *)calloc(ix->n_buckets + 1, sizeof(uint64_t));
    /* pass 1: occurrences per bucket */
    for (uint32_t s = 0; s < n_seqs; ++s) {
        uint64_t L = seq_start[s + 1] - seq_start[s];
        const uint8_t *seq = bases + seq_start[s];
        for (uint64_t pos = 0; pos + (uint64_t)span <= L; pos += (uint64_t)t) {
            int64_t c = seed_code(seq + pos, ix->mask, span);
            if (c >= 0) ix->bucket_start[c + 1]++;
        }
    }
    for (uint64_t c = 0; c < ix->n_buckets; ++c) ix->bucket_start[c + 1] += ix->bucket_start[c];
    ix->n_postings = ix->bucket_start[ix->n_buckets];
    ix->post_seq = (uint32_t *)malloc(sizeof(uint32_t) * (ix->n_postings ? ix->n_postings : 1));
    ix->post_pos = (uint32_t *)malloc(sizeof(uint32_t) * (ix->n_postings ? ix->n_postings : 1));
    /* pass 2: place occurrences in bank order (stable, so each bucket is sorted) */
    uint64_t *cursor = (uint64_t *)malloc(sizeof(uint64_t) * ix->n_buckets);
    memcpy(cursor, ix->bucket_start, sizeof(uint64_t) * ix->n_buckets);
    for (uint32_t s = 0; s < n_seqs; ++s) {
        uint64_t L = seq_start[s + 1] - seq_start[s];
        const uint8_t *seq = bases + seq_start[s];
        for (uint64_t pos = 0; pos + (uint64_t)span <= L; pos += (uint64_t)t) {
            int64_t c = seed_code(seq + pos, ix->mask, span);
            if (c < 0) continue;
            uint64_t at = cursor[c]++;
            ix->post_seq[at] = s;
            ix->post_pos[at] = (uint32_t)pos;
        }
    }
    free(cursor);
    return ix;
}

/* Marks in keep[] (4^k bytes) the code of every seed of a query (offsets 0 .. m - span,
 * seeds holding a non-base at a kept position excepted), as the search looks them up. */
void or_mark_query_codes(const uint8_t *q, uint32_t m, const char *mask, uint8_t *keep) {
    int span = (int)strlen(mask);
    for (uint64_t x = 0; x + (uint64_t)span <= m; ++x) {
        int64_t c = seed_code(q + x, mask, span);
        if (c >= 0) keep[c] = 1;
    }
}

typedef struct {
    const uint8_t *bases;
    const uint64_t *seq_start;
    uint32_t s_lo, s_hi;
    const char *mask;
    int span, t;
    const uint8_t *keep;
    uint64_t n, cap;
    uint64_t *code;
    uint32_t *seq, *pos;
} restrict_scan;

static void *restrict_scan_run(void *arg) {
    restrict_scan *r = (restrict_scan *)arg;
    for (uint32_t s = r->s_lo; s < r->s_hi; ++s) {
        uint64_t L = r->seq_start[s + 1] - r->seq_start[s];
        const uint8_t *seq = r->bases + r->seq_start[s];
        for (uint64_t pos = 0; pos + (uint64_t)r->span <= L; pos += (uint64_t)r->t) {
            int64_t c = seed_code(seq + pos, r->mask, r->span);
            if (c < 0 || !r->keep[c]) continue;
            if (r->n == r->cap) {
                r->cap = r->cap ? 2 * r->cap : 1024;
                r->code = (uint64_t *)realloc(r->code, sizeof(uint64_t) * r->cap);
                r->seq = (uint32_t *)realloc(r->seq, sizeof(uint32_t) * r->cap);
                r->pos = (uint32_t *)realloc(r->pos, sizeof(uint32_t) * r->cap);
            }
            r->code[r->n] = (uint64_t)c; r->seq[r->n] = s; r->pos[r->n] = (uint32_t)pos;
            ++r->n;
        }
    }
    return NULL;
}

/* The index restricted to the buckets whose code has keep[code] != 0: each of them holds
 * exactly the occurrences of the full index in the same (sequence, position) order, the
 * others are empty.  A query whose seed codes are all kept is therefore searched exactly
 * as against the full index.  It serves tests on banks whose full index would not fit
 * the host.  The bank is scanned by `threads` threads over consecutive sequence ranges;
 * their occurrences, taken range by range, are in bank order. */
or_index *or_index_build_restricted(const uint8_t *bases, const uint64_t *seq_start, uint32_t n_seqs,
                                    const char *mask, int t, const uint8_t *keep, int threads) {
    or_index *ix = or_index_build_masked(bases, seq_start, 0, mask, t);  /* validated, empty */
    if (!ix) return NULL;
    ix->n_seqs = n_seqs;
    if (threads < 1) threads = 1;
    if ((uint32_t)threads > n_seqs) threads = n_seqs ? (int)n_seqs : 1;
    restrict_scan *rs = (restrict_scan *)calloc((size_t)threads, sizeof(restrict_scan));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int i = 0; i < threads; ++i) {
        rs[i].bases = bases; rs[i].seq_start = seq_start; rs[i].mask = ix->mask; rs[i].span = ix->span;
        rs[i].t = t; rs[i].keep = keep;
        rs[i].s_lo = (uint32_t)((uint64_t)n_seqs * i / threads);
        rs[i].s_hi = (uint32_t)((uint64_t)n_seqs * (i + 1) / threads);
        pthread_create(&th[i], NULL, restrict_scan_run, &rs[i]);
    }
    for (int i = 0; i < threads; ++i) pthread_join(th[i], NULL);
    uint64_t total = 0;
    for (int i = 0; i < threads; ++i) {
        total += rs[i].n;
        for (uint64_t j = 0; j < rs[i].n; ++j) ix->bucket_start[rs[i].code[j] + 1]++;
    }
    for (uint64_t c = 0; c < ix->n_buckets; ++c) ix->bucket_start[c + 1] += ix->bucket_start[c];
    ix->n_postings = total;
    free(ix->post_seq); free(ix->post_pos);
    ix->post_seq = (uint32_t *)malloc(sizeof(uint32_t) * (total ? total : 1));
    ix->post_pos = (uint32_t *)malloc(sizeof(uint32_t) * (total ? total : 1));
    uint64_t *cursor = (uint64_t *)malloc(sizeof(uint64_t) * ix->n_buckets);
    memcpy(cursor, ix->bucket_start, sizeof(uint64_t) * ix->n_buckets);
    for (int i = 0; i < threads; ++i) {
        for (uint64_t j = 0; j < rs[i].n; ++j) {
            uint64_t at = cursor[rs[i].code[j]]++;
            ix->post_seq[at] = rs[i].seq[j];
            ix->post_pos[at] = rs[i].pos[j];
        }
        free(rs[i].code); free(rs[i].seq); free(rs[i].pos);
    }
    free(cursor); free(rs); free(th);
    return ix;
}

/* plain k-base windows: the mask of k ones */
or_index *or_index_build(const uint8_t *bases, const uint64_t *seq_start, uint32_t n_seqs, int k, int t) {
    if (k < 1 || k > 16) return NULL;
    char mask[33];
    memset(mask, '1', (size_t)k);
    mask[k] = 0;
    return or_index_build_masked(bases, seq_start, n_seqs, mask, t);
}

void or_index_free(or_index *ix) {
    if (!ix) return;
    free(ix->bucket_start); free(ix->post_seq); free(ix->post_pos); free(ix);
}

uint64_t or_index_n_postings(const or_index *ix) { return ix->n_postings; }
const uint64_t *or_index_bucket_start(const or_index *ix) { return ix->bucket_start; }
const uint32_t *or_index_post_seq(const or_index *ix) { return ix->post_seq; }
const uint32_t *or_index_post_pos(const or_index *ix) { return ix->post_pos; }

/* ------------------------------------------------------------ records --- */
typedef struct {
    int32_t match, mismatch, gap_open, gap_extend; /* scores: +1, -3, -5, -2 */
    double lambda, K;
    uint32_t max_hit_distance;   /* D: largest query-position gap inside one HSP */
    uint32_t min_hsp_len;
    int32_t xdrop;
    uint32_t max_alignments;     /* 0 = all */
    uint32_t band_w;
    double max_evalue;           /* INFINITY = no filter */
    int32_t keep_hits;           /* export the sorted hit list */
} or_params;

typedef struct { uint32_t qpos, seq, pos; } or_hit;
typedef struct { uint32_t seq, qs, qe, ds, de, len; } or_hsp;
typedef struct {
    uint32_t seq, qs, qe, ds, de;
    int32_t score;
    uint32_t rank, pad;
    double evalue, bits;
} or_aln;

typedef struct {
    uint64_t n_hits;
    or_hit *hits; uint64_t n_hits_kept;
    or_hsp *hsp; uint32_t n_hsp;        /* HSPs from merged hits, (seq, diagonal, qs) order */
    or_hsp *ext; uint32_t n_ext;        /* the same HSPs after extension */
    or_hsp *merged; uint32_t n_merged;  /* after merging overlapped HSPs, sweep order */
    or_hsp *sel; uint32_t n_sel;        /* selected, longest first */
    or_aln *aln; uint32_t n_aln;        /* banded Smith-Waterman of each selected HSP */
    or_aln *ranked; uint32_t n_ranked;  /* final list, best score first */
    int32_t status;
} or_result;

void or_result_free(or_result *r) {
    if (!r) return;
    free(r->hits); free(r->hsp); free(r->ext); free(r->merged); free(r->sel); free(r->aln); free(r->ranked);
    memset(r, 0, sizeof(*r));
}

/* ------------------------------------------------- phase 2: hits -> HSP --- */
static int cmp_hit(const void *a, const void *b) {
    const or_hit *x = (const or_hit *)a, *y = (const or_hit *)b;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    int64_t dx = (int64_t)x->pos - x->qpos, dy = (int64_t)y->pos - y->qpos;
    if (dx != dy) return dx < dy ? -1 : 1;
    if (x->qpos != y->qpos) return x->qpos < y->qpos ? -1 : 1;
    return 0;
}

/* "Searching process", phase 2: every encoded query window is looked up; the
 * occurrences are grouped per bank sequence (here: per sequence and diagonal),
 * occurrences closer than D along the query are merged into one area, and areas
 * shorter than the minimum HSP length are dropped.  An area runs from its first
 * seed to the end of its last one (a seed covers `span` bases).  HSP length is
 * the smaller of its query and bank spans. */
static void find_hsps(const or_index *ix, const uint8_t *q, uint32_t m, const or_params *p, or_result *r) {
    int span = ix->span; /* a seed covers span bases (k without a mask) */
    uint64_t nh = 0, cap = 1024;
    or_hit *hits = (or_hit *)malloc(sizeof(or_hit) * cap);
    for (uint32_t qpos = 0; qpos + (uint32_t)span <= m; ++qpos) {
        int64_t c = seed_code(q + qpos, ix->mask, span);
        if (c < 0) continue;
        for (uint64_t e = ix->bucket_start[c]; e < ix->bucket_start[c + 1]; ++e) {
            if (nh == cap) { cap *= 2; hits = (or_hit *)realloc(hits, sizeof(or_hit) * cap); }
            hits[nh].qpos = qpos; hits[nh].seq = ix->post_seq[e]; hits[nh].pos = ix->post_pos[e];
            ++nh;
        }
    }
    r->n_hits = nh;
    qsort(hits, nh, sizeof(or_hit), cmp_hit);

    uint32_t cap_h = 64, n = 0;
    or_hsp *out = (or_hsp *)malloc(sizeof(or_hsp) * cap_h);
    uint64_t i = 0;
    while (i < nh) {
        uint64_t j = i; /* the chain is hits[i..j] */
        while (j + 1 < nh && hits[j + 1].seq == hits[i].seq &&
               (int64_t)hits[j + 1].pos - hits[j + 1].qpos == (int64_t)hits[i].pos - hits[i].qpos &&
               hits[j + 1].qpos - hits[j].qpos <= p->max_hit_distance)
            ++j;
        uint32_t qs = hits[i].qpos, qe = hits[j].qpos + (uint32_t)span;
        uint32_t ds = hits[i].pos, de = hits[j].pos + (uint32_t)span;
        uint32_t len = (qe - qs) < (de - ds) ? (qe - qs) : (de - ds);
        if (len >= p->min_hsp_len) {
            if (n == cap_h) { cap_h *= 2; out = (or_hsp *)realloc(out, sizeof(or_hsp) * cap_h); }
            or_hsp h = {hits[i].seq, qs, qe, ds, de, len};
            out[n++] = h;
        }
        i = j + 1;
    }
    r->hsp = out; r->n_hsp = n;
    if (p->keep_hits) { r->hits = hits; r->n_hits_kept = nh; }
    else free(hits);
}

/* ------------------------------------------------ phase 3: extension --- */
static int32_t pair_score(uint8_t a, uint8_t b, const or_params *p) {
    int ca = base_code(a), cb = base_code(b);
    return (ca >= 0 && ca == cb) ? p->match : p->mismatch;
}

/* "Searching process", phase 3: both ends of an HSP are pushed outwards, one
 * base pair at a time along the HSP's own diagonal, keeping a running score; the
 * walk stops at a sequence end or once the score has fallen more than X below
 * the best score seen, and the end moves to where the best score was (the first
 * such place).  The HSP interior is not rescored. */
void or_extend(const uint8_t *q, uint32_t m, const uint8_t *S, uint32_t L, const or_params *p, or_hsp *h) {
    int32_t score = 0, best = 0;
    uint32_t ext = 0;
    for (uint32_t e = 1; e <= h->qs && e <= h->ds; ++e) {
        score += pair_score(q[h->qs - e], S[h->ds - e], p);
        if (score > best) { best = score; ext = e; }
        else if (best - score > p->xdrop) break;
    }
    h->qs -= ext; h->ds -= ext;
    score = 0; best = 0; ext = 0;
    for (uint32_t e = 1; h->qe + e - 1 < m && h->de + e - 1 < L; ++e) {
        score += pair_score(q[h->qe + e - 1], S[h->de + e - 1], p);
        if (score > best) { best = score; ext = e; }
        else if (best - score > p->xdrop) break;
    }
    h->qe += ext; h->de += ext;
    h->len = (h->qe - h->qs) < (h->de - h->ds) ? (h->qe - h->qs) : (h->de - h->ds);
}

/* ------------------------------------------- phase 4: overlapped HSPs --- */
static int cmp_sweep(const void *a, const void *b) {
    const or_hsp *x = (const or_hsp *)a, *y = (const or_hsp *)b;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    if (x->qs != y->qs) return x->qs < y->qs ? -1 : 1;
    if (x->ds != y->ds) return x->ds < y->ds ? -1 : 1;
    if (x->qe != y->qe) return x->qe < y->qe ? -1 : 1;
    if (x->de != y->de) return x->de < y->de ? -1 : 1;
    return 0;
}

/* "Searching process", phase 4: HSPs of one bank sequence whose query areas
 * intersect and whose bank areas intersect are merged into one HSP covering
 * both.  Single sweep in (qs, ds, qe, de) order; each HSP joins the current box
 * or starts a new one.  Sorts `in` in place; writes the boxes to out. */
uint32_t or_merge_overlaps(or_hsp *in, uint32_t n, or_hsp *out) {
    qsort(in, n, sizeof(or_hsp), cmp_sweep);
    uint32_t no = 0;
    uint32_t i = 0;
    while (i < n) {
        or_hsp box = in[i];
        uint32_t j = i + 1;
        while (j < n && in[j].seq == box.seq) {
            const or_hsp *h = &in[j];
            int q_meet = h->qs < box.qe && box.qs < h->qe;
            int d_meet = h->ds < box.de && box.ds < h->de;
            if (!(q_meet && d_meet)) break;
            if (h->qs < box.qs) box.qs = h->qs;
            if (h->qe > box.qe) box.qe = h->qe;
            if (h->ds < box.ds) box.ds = h->ds;
            if (h->de > box.de) box.de = h->de;
            ++j;
        }
        box.len = (box.qe - box.qs) < (box.de - box.ds) ? (box.qe - box.qs) : (box.de - box.ds);
        out[no++] = box;
        i = j;
    }
    return no;
}

/* ---------------------------------------------- phase 5: selection --- */
static int cmp_length(const void *a, const void *b) {
    const or_hsp *x = (const or_hsp *)a, *y = (const or_hsp *)b;
    if (x->len != y->len) return x->len > y->len ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    if (x->qs != y->qs) return x->qs < y->qs ? -1 : 1;
    if (x->ds != y->ds) return x->ds < y->ds ? -1 : 1;
    if (x->qe != y->qe) return x->qe < y->qe ? -1 : 1;
    if (x->de != y->de) return x->de < y->de ? -1 : 1;
    return 0;
}

/* ------------------------------------- phase 6: banded Smith-Waterman --- */
/* "Searching process", phase 6: local alignment (Smith-Waterman with affine
 * gaps, Gotoh's three-state form) restricted to the cells near the HSP's
 * diagonals.  The DP covers rows [qs-w, qe+w) x columns [ds-w, de+w) clipped to
 * the sequences, and only the diagonals j-i in [min(ds-qs, de-qe)-w,
 * max(ds-qs, de-qe)+w].  A gap of length g scores gap_open + g*gap_extend.
 *   E(i,j) = max(H(i-1,j) + go + ge, E(i-1,j) + ge)      (open wins ties)
 *   F(i,j) = max(H(i,j-1) + go + ge, F(i,j-1) + ge)      (open wins ties)
 *   H(i,j) = max(0, H(i-1,j-1) + s(i,j), E(i,j), F(i,j)) (diagonal, then E, then F on ties)
 * A neighbour outside the DP region has H = 0 and E = F = -infinity, so an
 * alignment may begin at any cell of the region.  Each state carries the cell
 * where its alignment began; a diagonal step from H <= 0 begins at this cell.
 * The reported alignment ends at the best cell (largest H, then smallest i, then
 * smallest j) and the ranges are half-open. */
void or_banded_sw(const uint8_t *q, uint32_t m, const uint8_t *S, uint32_t L, const or_hsp *h,
                  const or_params *p, or_aln *out) {
    const int64_t w = p->band_w;
    const int32_t go = p->gap_open, ge = p->gap_extend;
    int64_t d_s = (int64_t)h->ds - h->qs, d_e = (int64_t)h->de - h->qe;
    int64_t dlo = (d_s < d_e ? d_s : d_e) - w, dhi = (d_s > d_e ? d_s : d_e) + w;
    int64_t I0 = (int64_t)h->qs - w, I1 = (int64_t)h->qe + w;
    int64_t J0 = (int64_t)h->ds - w, J1 = (int64_t)h->de + w;
    if (I0 < 0) I0 = 0;
    if (J0 < 0) J0 = 0;
    if (I1 > (int64_t)m) I1 = m;
    if (J1 > (int64_t)L) J1 = L;
    memset(out, 0, sizeof(*out));
    out->seq = h->seq;
    if (I1 <= I0 || J1 <= J0) return;
    int64_t W = J1 - J0;
    /* two full-width rows: [0] = previous row, [1] = current row */
    int32_t *H[2], *E[2], *F[2];
    int64_t *SHi[2], *SHj[2], *SEi[2], *SEj[2], *SFi[2], *SFj[2];
    for (int r = 0; r < 2; ++r) {
        H[r] = (int32_t *)calloc(W, 4); E[r] = (int32_t *)calloc(W, 4); F[r] = (int32_t *)calloc(W, 4);
        SHi[r] = (int64_t *)calloc(W, 8); SHj[r] = (int64_t *)calloc(W, 8);
        SEi[r] = (int64_t *)calloc(W, 8); SEj[r] = (int64_t *)calloc(W, 8);
        SFi[r] = (int64_t *)calloc(W, 8); SFj[r] = (int64_t *)calloc(W, 8);
    }
#define IN_DP(ii, jj) ((ii) >= I0 && (ii) < I1 && (jj) >= J0 && (jj) < J1 && (jj) - (ii) >= dlo && (jj) - (ii) <= dhi)
    int32_t best = 0;
    int64_t bi = -1, bj = -1, bsi = -1, bsj = -1;
    int cur = 1, prv = 0;
    for (int64_t i = I0; i < I1; ++i) {
        int64_t jlo = i + dlo > J0 ? i + dlo : J0;
        int64_t jhi = i + dhi < J1 - 1 ? i + dhi : J1 - 1;
        for (int64_t j = jlo; j <= jhi; ++j) {
            int64_t x = j - J0;
            int32_t e, f, hv;
            int64_t sei = 0, sej = 0, sfi = 0, sfj = 0, shi, shj;
            if (IN_DP(i - 1, j)) {
                int32_t eo = H[prv][x] + go + ge, ee = E[prv][x] + ge;
                if (eo >= ee) { e = eo; sei = SHi[prv][x]; sej = SHj[prv][x]; }
                else { e = ee; sei = SEi[prv][x]; sej = SEj[prv][x]; }
            } else {
                e = OR_NEG;
            }
            if (IN_DP(i, j - 1)) {
                int32_t fo = H[cur][x - 1] + go + ge, fe = F[cur][x - 1] + ge;
                if (fo >= fe) { f = fo; sfi = SHi[cur][x - 1]; sfj = SHj[cur][x - 1]; }
                else { f = fe; sfi = SFi[cur][x - 1]; sfj = SFj[cur][x - 1]; }
            } else {
                f = OR_NEG;
            }
            int32_t hd = 0;
            int64_t sdi = i, sdj = j;
            if (IN_DP(i - 1, j - 1)) {
                hd = H[prv][x - 1];
                if (hd > 0) { sdi = SHi[prv][x - 1]; sdj = SHj[prv][x - 1]; }
            }
            int32_t dg = hd + pair_score(q[i], S[j], p);
            if (dg >= e && dg >= f && dg > 0) { hv = dg; shi = sdi; shj = sdj; }
            else if (e >= f && e > 0) { hv = e; shi = sei; shj = sej; }
            else if (f > 0) { hv = f; shi = sfi; shj = sfj; }
            else { hv = 0; shi = i; shj = j; }
            H[cur][x] = hv; E[cur][x] = e; F[cur][x] = f;
            SHi[cur][x] = shi; SHj[cur][x] = shj;
            SEi[cur][x] = sei; SEj[cur][x] = sej;
            SFi[cur][x] = sfi; SFj[cur][x] = sfj;
            if (hv > best) { best = hv; bi = i; bj = j; bsi = shi; bsj = shj; }
        }
        cur ^= 1; prv ^= 1;
    }
#undef IN_DP
    for (int r = 0; r < 2; ++r) {
        free(H[r]); free(E[r]); free(F[r]); free(SHi[r]); free(SHj[r]);
        free(SEi[r]); free(SEj[r]); free(SFi[r]); free(SFj[r]);
    }
    if (best > 0) {
        out->qs = (uint32_t)bsi; out->qe = (uint32_t)(bi + 1);
        out->ds = (uint32_t)bsj; out->de = (uint32_t)(bj + 1);
        out->score = best;
    }
}

/* ---------------------------------------- phase 7: ranking, statistics --- */
/* Karlin-Altschul statistics: E = K m n exp(-lambda S) with m the query length
 * and n the bank length in bases; bit score = (lambda S - ln K) / ln 2. */
double or_evalue(int32_t score, double m, double n, const or_params *p) {
    return p->K * m * n * exp(-p->lambda * (double)score);
}

double or_bits(int32_t score, const or_params *p) {
    return (p->lambda * (double)score - log(p->K)) / log(2.0);
}

static int cmp_score(const void *a, const void *b) {
    const or_aln *x = (const or_aln *)a, *y = (const or_aln *)b;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
    if (x->qs != y->qs) return x->qs < y->qs ? -1 : 1;
    if (x->ds != y->ds) return x->ds < y->ds ? -1 : 1;
    if (x->qe != y->qe) return x->qe < y->qe ? -1 : 1;
    if (x->de != y->de) return x->de < y->de ? -1 : 1;
    return 0;
}

/* "Searching process", phase 7: alignments sorted by score (ties: sequence,
 * query start, bank start, query end, bank end), alignments with the same
 * sequence and ranges as an earlier one removed (the earlier, better one is
 * kept), e-value and bit score attached, e-value cut applied, ranks numbered
 * from 0.  Writes to out (capacity n); returns the count. */
uint32_t or_rank(const or_aln *in, uint32_t n, double m, double n_bank, const or_params *p, or_aln *out) {
    or_aln *all = (or_aln *)malloc(sizeof(or_aln) * (n ? n : 1));
    uint32_t na = 0;
    for (uint32_t i = 0; i < n; ++i)
        if (in[i].score > 0) all[na++] = in[i];
    qsort(all, na, sizeof(or_aln), cmp_score);
    uint32_t nr = 0;
    for (uint32_t i = 0; i < na; ++i) {
        int dup = 0;
        for (uint32_t j = 0; j < i && !dup; ++j) {
            const or_aln *a = &all[j], *b = &all[i];
            dup = a->seq == b->seq && a->qs == b->qs && a->qe == b->qe && a->ds == b->ds && a->de == b->de;
        }
        if (dup) continue;
        or_aln a = all[i];
        a.evalue = or_evalue(a.score, m, n_bank, p);
        a.bits = or_bits(a.score, p);
        if (!(a.evalue <= p->max_evalue)) continue;
        a.rank = nr;
        out[nr++] = a;
    }
    free(all);
    return nr;
}

/* ------------------------------------------------------------ search --- */
/* One query through the seven phases of "Searching process". */
int or_search_one(const or_index *ix, const uint8_t *q, uint32_t m, const or_params *p, or_result *r) {
    memset(r, 0, sizeof(*r));
    /* phases 1-2: input processing, index lookup, HSP construction */
    find_hsps(ix, q, m, p, r);
    /* phase 3: extension */
    r->ext = (or_hsp *)malloc(sizeof(or_hsp) * (r->n_hsp ? r->n_hsp : 1));
    for (uint32_t i = 0; i < r->n_hsp; ++i) {
        or_hsp h = r->hsp[i];
        const uint8_t *S = ix->bases + ix->seq_start[h.seq];
        uint32_t L = (uint32_t)(ix->seq_start[h.seq + 1] - ix->seq_start[h.seq]);
        or_extend(q, m, S, L, p, &h);
        r->ext[i] = h;
    }
    r->n_ext = r->n_hsp;
    /* phase 4: merge overlapped HSPs */
    or_hsp *tmp = (or_hsp *)malloc(sizeof(or_hsp) * (r->n_ext ? r->n_ext : 1));
    memcpy(tmp, r->ext, sizeof(or_hsp) * r->n_ext);
    r->merged = (or_hsp *)malloc(sizeof(or_hsp) * (r->n_ext ? r->n_ext : 1));
    r->n_merged = or_merge_overlaps(tmp, r->n_ext, r->merged);
    free(tmp);
    /* phase 5: longest first, at most max_alignments (0 = all) */
    r->sel = (or_hsp *)malloc(sizeof(or_hsp) * (r->n_merged ? r->n_merged : 1));
    memcpy(r->sel, r->merged, sizeof(or_hsp) * r->n_merged);
    qsort(r->sel, r->n_merged, sizeof(or_hsp), cmp_length);
    r->n_sel = r->n_merged;
    if (p->max_alignments && r->n_sel > p->max_alignments) r->n_sel = p->max_alignments;
    /* phase 6: banded local alignment of each selected HSP */
    r->aln = (or_aln *)malloc(sizeof(or_aln) * (r->n_sel ? r->n_sel : 1));
    for (uint32_t i = 0; i < r->n_sel; ++i) {
        const or_hsp *h = &r->sel[i];
        const uint8_t *S = ix->bases + ix->seq_start[h->seq];
        uint32_t L = (uint32_t)(ix->seq_start[h->seq + 1] - ix->seq_start[h->seq]);
        or_banded_sw(q, m, S, L, h, p, &r->aln[i]);
    }
    r->n_aln = r->n_sel;
    /* phase 7: best score first, exact duplicates removed, statistics */
    r->ranked = (or_aln *)malloc(sizeof(or_aln) * (r->n_aln ? r->n_aln : 1));
    r->n_ranked = or_rank(r->aln, r->n_aln, (double)m, (double)ix->seq_start[ix->n_seqs], p, r->ranked);
    return 0;
}

/* ------------------------------------------- many queries, many threads --- */
typedef struct {
    const or_index *ix;
    const uint8_t *qbases;
    const uint64_t *qstart;
    uint32_t nq;
    const or_params *p;
    or_result *res;
    uint32_t *next;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *j = (batch_job *)arg;
    for (;;) {
        uint32_t i = __atomic_fetch_add(j->next, 1, __ATOMIC_RELAXED);
        if (i >= j->nq) break;
        or_search_one(j->ix, j->qbases + j->qstart[i], (uint32_t)(j->qstart[i + 1] - j->qstart[i]), j->p,
                      &j->res[i]);
    }
    return NULL;
}

/* Searches nq queries; each query is independent, so threads take whole queries. */
int or_search_batch(const or_index *ix, const uint8_t *qbases, const uint64_t *qstart, uint32_t nq,
                    const or_params *p, int n_threads, or_result *res) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    uint32_t next = 0;
    batch_job job = {ix, qbases, qstart, nq, p, res, &next};
    if (n_threads == 1) { batch_worker(&job); return 0; }
    pthread_t th[256];
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, batch_worker, &job);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    return 0;
}

void or_result_free_batch(or_result *res, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i) or_result_free(&res[i]);
}

size_t or_sizeof_result(void) { return sizeof(or_result); }
size_t or_sizeof_params(void) { return sizeof(or_params); }
size_t or_sizeof_aln(void) { return sizeof(or_aln); }
