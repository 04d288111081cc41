/*
 * synth.c - seeded synthetic DNA workloads shaped like the paper's experiments.
 *
 * The paper measures on hs_phase3 + six RefSeq banks (4.25 Gbp, Results section)
 * and on query sets made of one bank sequence plus mutated copies of it.  Those
 * data are not available, so every workload here is generated from a seed.
 *
 * This file holds NO arithmetic of the search method (no k-mer codes, no
 * scoring, no index).  It only draws random sequences; the CUDA path and the
 * CPU oracle both consume its output.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018), each stream seeded by
 * splitmix64 (Steele, Lea & Flood, 2014) from (seed, purpose, item index), so a
 * sequence's bases do not depend on how many threads filled the bank.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG --- */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t purpose, uint64_t item) {
    uint64_t x = seed;
    uint64_t a = splitmix64_next(&x);
    x = a ^ (purpose * 0xD1B54A32D192ED03ULL);
    uint64_t b = splitmix64_next(&x);
    x = b ^ (item * 0x8CB92BA72F3D8DD7ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform double in [0,1) with 53 random bits */
static inline double rng_unif(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n) (multiply-shift; bias < 2^-32 for n < 2^32) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static double rng_normal(rng_t *r) { /* Box-Muller, one value per call */
    double u1 = rng_unif(r), u2 = rng_unif(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

/* one base with G+C probability gc (G and C equally likely, A and T equally likely) */
static inline char draw_base(rng_t *r, double gc) {
    double u = rng_unif(r);
    if (u < gc) return (u < 0.5 * gc) ? 'G' : 'C';
    return (u < gc + 0.5 * (1.0 - gc)) ? 'A' : 'T';
}

static inline char other_base(rng_t *r, char b) {
    char c;
    do { c = BASES[rng_below(r, 4)]; } while (c == b);
    return c;
}

/* purposes (independent streams) */
enum { P_LEN = 1, P_GC = 2, P_BASES = 3, P_FAM = 4, P_REPEAT = 5, P_QLEN = 6, P_QUERY = 7, P_ARRIVAL = 8 };

/* ---------------------------------------------------------- bank spec --- */
typedef struct {
    uint64_t seed;
    uint32_t n_seqs;
    int32_t len_dist;        /* 0: uniform [len_lo, len_hi]; 1: log-normal(median, sigma) clipped */
    double len_median, len_sigma;
    uint32_t len_lo, len_hi;
    double gc_lo, gc_hi;     /* per-sequence GC content ~ U[gc_lo, gc_hi] */
    uint32_t n_families;     /* repeat families (0 = none) */
    uint32_t fam_len_lo, fam_len_hi;   /* consensus length, log-uniform */
    double fam_div_lo, fam_div_hi;     /* per-copy divergence ~ U[lo, hi] */
    double repeat_frac;      /* stop planting copies once this fraction of bases was overwritten */
    int32_t n_threads;
} synth_bank_spec;

static uint32_t draw_len(rng_t *r, const synth_bank_spec *sp) {
    double L;
    if (sp->len_dist == 0) {
        L = (double)sp->len_lo + (double)rng_below(r, (uint64_t)(sp->len_hi - sp->len_lo) + 1);
    } else {
        L = floor(sp->len_median * exp(sp->len_sigma * rng_normal(r)) + 0.5);
        if (L < sp->len_lo) L = sp->len_lo;
        if (L > sp->len_hi) L = sp->len_hi;
    }
    return (uint32_t)L;
}

/* Fills seq_start[0..n_seqs] (exclusive prefix of lengths).  Returns total bases. */
uint64_t synth_bank_layout(const synth_bank_spec *sp, uint64_t *seq_start) {
    rng_t r;
    rng_init(&r, sp->seed, P_LEN, 0);
    uint64_t acc = 0;
    for (uint32_t s = 0; s < sp->n_seqs; ++s) {
        seq_start[s] = acc;
        acc += draw_len(&r, sp);
    }
    seq_start[sp->n_seqs] = acc;
    return acc;
}

typedef struct {
    const synth_bank_spec *sp;
    const uint64_t *seq_start;
    char *bases;
    uint32_t s0, s1;
} fill_job;

static void *fill_worker(void *arg) {
    fill_job *j = (fill_job *)arg;
    for (uint32_t s = j->s0; s < j->s1; ++s) {
        rng_t rg, rb;
        rng_init(&rg, j->sp->seed, P_GC, s);
        double gc = j->sp->gc_lo + (j->sp->gc_hi - j->sp->gc_lo) * rng_unif(&rg);
        rng_init(&rb, j->sp->seed, P_BASES, s);
        char *dst = j->bases + j->seq_start[s];
        uint64_t L = j->seq_start[s + 1] - j->seq_start[s];
        for (uint64_t i = 0; i < L; ++i) dst[i] = draw_base(&rb, gc);
    }
    return NULL;
}

/* Writes a mutated copy of src[0..n) into dst (capacity cap); returns bases written.
 * Per source base: with probability p_sub it is substituted, with probability p_indel
 * an indel happens (half insertions of a random base before it, half deletions). */
static uint64_t mutate_copy(rng_t *r, const char *src, uint64_t n, double p_sub, double p_indel,
                            char *dst, uint64_t cap) {
    uint64_t w = 0;
    for (uint64_t i = 0; i < n && w < cap; ++i) {
        double u = rng_unif(r);
        if (u < p_indel) {
            if (rng_unif(r) < 0.5) {              /* insertion, then the base itself */
                dst[w++] = BASES[rng_below(r, 4)];
                if (w < cap) dst[w++] = src[i];
            }                                      /* else deletion: skip src[i] */
        } else if (u < p_indel + p_sub) {
            dst[w++] = other_base(r, src[i]);
        } else {
            dst[w++] = src[i];
        }
    }
    return w;
}

/* Fills bases[seq_start[0] .. seq_start[n_seqs]) and plants repeat copies. */
void synth_bank_fill(const synth_bank_spec *sp, const uint64_t *seq_start, char *bases) {
    int nt = sp->n_threads > 0 ? sp->n_threads : 1;
    if (nt > 64) nt = 64;
    pthread_t th[64];
    fill_job jobs[64];
    uint32_t per = (sp->n_seqs + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        jobs[t].sp = sp; jobs[t].seq_start = seq_start; jobs[t].bases = bases;
        jobs[t].s0 = (uint32_t)((uint64_t)t * per < sp->n_seqs ? (uint64_t)t * per : sp->n_seqs);
        jobs[t].s1 = (uint32_t)((uint64_t)(t + 1) * per < sp->n_seqs ? (uint64_t)(t + 1) * per : sp->n_seqs);
        pthread_create(&th[t], NULL, fill_worker, &jobs[t]);
    }
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);

    if (sp->n_families == 0 || sp->repeat_frac <= 0.0) return;
    /* repeat families: consensus sequences with uniform bases */
    uint32_t nf = sp->n_families;
    char **fam = (char **)malloc(sizeof(char *) * nf);
    uint32_t *flen = (uint32_t *)malloc(sizeof(uint32_t) * nf);
    for (uint32_t f = 0; f < nf; ++f) {
        rng_t r;
        rng_init(&r, sp->seed, P_FAM, f);
        double lo = log((double)sp->fam_len_lo), hi = log((double)sp->fam_len_hi);
        flen[f] = (uint32_t)floor(exp(lo + (hi - lo) * rng_unif(&r)) + 0.5);
        fam[f] = (char *)malloc(flen[f]);
        for (uint32_t i = 0; i < flen[f]; ++i) fam[f][i] = BASES[rng_below(&r, 4)];
    }
    uint64_t total = seq_start[sp->n_seqs];
    uint64_t budget = (uint64_t)(sp->repeat_frac * (double)total);
    uint64_t written = 0;
    rng_t r;
    rng_init(&r, sp->seed, P_REPEAT, 0);
    uint64_t guard = 0;
    while (written < budget && guard++ < (uint64_t)1 << 40) {
        uint32_t f = (uint32_t)rng_below(&r, nf);
        double div = sp->fam_div_lo + (sp->fam_div_hi - sp->fam_div_lo) * rng_unif(&r);
        uint64_t at = rng_below(&r, total);
        /* containing sequence: binary search */
        uint32_t lo = 0, hi = sp->n_seqs;
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (seq_start[mid] <= at) lo = mid; else hi = mid;
        }
        uint64_t cap = seq_start[lo + 1] - at;
        written += mutate_copy(&r, fam[f], flen[f], div * 5.0 / 6.0, div / 6.0, bases + at, cap);
    }
    for (uint32_t f = 0; f < nf; ++f) free(fam[f]);
    free(fam); free(flen);
}

/* -------------------------------------------------------- query spec --- */
typedef struct {
    uint64_t seed;
    uint32_t n_queries;
    int32_t len_dist;        /* 0: uniform [len_lo, len_hi]; 1: log-uniform */
    uint32_t len_lo, len_hi;
    double homolog_frac;     /* fraction of queries copied (with mutations) from the bank */
    double div_lo, div_hi;   /* homolog divergence ~ U[div_lo, div_hi] (used when p_sub < 0) */
    double p_sub, p_indel;   /* fixed per-base rates; p_sub < 0 selects the divergence model */
    double random_gc;        /* GC content of non-homolog (random) queries */
} synth_query_spec;

/* Query lengths before mutation, and the per-query source (written to meta[5*i ...]:
 * is_homolog, src_seq, src_pos, src_len, divergence*1e6).  Returns the capacity
 * needed for the bases (an upper bound; the true total comes from synth_queries_fill). */
uint64_t synth_queries_plan(const synth_query_spec *qs, const uint64_t *seq_start, uint32_t n_seqs,
                            uint64_t *meta) {
    rng_t r;
    rng_init(&r, qs->seed, P_QLEN, 0);
    uint64_t cap = 0;
    uint32_t maxlen = 0;
    for (uint32_t s = 0; s < n_seqs; ++s) {
        uint64_t L = seq_start[s + 1] - seq_start[s];
        if (L > maxlen) maxlen = (uint32_t)L;
    }
    for (uint32_t i = 0; i < qs->n_queries; ++i) {
        uint32_t len;
        if (qs->len_dist == 0) {
            len = qs->len_lo + (uint32_t)rng_below(&r, (uint64_t)(qs->len_hi - qs->len_lo) + 1);
        } else {
            double lo = log((double)qs->len_lo), hi = log((double)qs->len_hi);
            len = (uint32_t)floor(exp(lo + (hi - lo) * rng_unif(&r)) + 0.5);
        }
        int hom = rng_unif(&r) < qs->homolog_frac;
        uint64_t src_seq = 0, src_pos = 0;
        double div = 0.0;
        if (hom) {
            if (len > maxlen) len = maxlen;
            for (;;) { /* a sequence at least as long as the query, uniformly */
                src_seq = rng_below(&r, n_seqs);
                uint64_t L = seq_start[src_seq + 1] - seq_start[src_seq];
                if (L >= len) { src_pos = rng_below(&r, L - len + 1); break; }
            }
            div = qs->div_lo + (qs->div_hi - qs->div_lo) * rng_unif(&r);
        }
        meta[5 * (uint64_t)i + 0] = (uint64_t)hom;
        meta[5 * (uint64_t)i + 1] = src_seq;
        meta[5 * (uint64_t)i + 2] = src_pos;
        meta[5 * (uint64_t)i + 3] = len;
        meta[5 * (uint64_t)i + 4] = (uint64_t)floor(div * 1e6 + 0.5);
        cap += 2 * (uint64_t)len + 1; /* insertions can at most double a copy */
    }
    return cap;
}

/* Writes queries back to back into out (capacity cap) and their starts into start[0..n]. */
uint64_t synth_queries_fill(const synth_query_spec *qs, const uint64_t *meta, const uint64_t *seq_start,
                            const char *bank, char *out, uint64_t cap, uint64_t *start) {
    uint64_t w = 0;
    for (uint32_t i = 0; i < qs->n_queries; ++i) {
        rng_t r;
        rng_init(&r, qs->seed, P_QUERY, i);
        start[i] = w;
        uint64_t len = meta[5 * (uint64_t)i + 3];
        if (meta[5 * (uint64_t)i + 0]) {
            const char *src = bank + seq_start[meta[5 * (uint64_t)i + 1]] + meta[5 * (uint64_t)i + 2];
            double p_sub, p_indel;
            if (qs->p_sub >= 0.0) { p_sub = qs->p_sub; p_indel = qs->p_indel; }
            else {
                double div = (double)meta[5 * (uint64_t)i + 4] * 1e-6;
                p_sub = div * 5.0 / 6.0; p_indel = div / 6.0;
            }
            w += mutate_copy(&r, src, len, p_sub, p_indel, out + w, cap - w);
        } else {
            for (uint64_t j = 0; j < len && w < cap; ++j) out[w++] = draw_base(&r, qs->random_gc);
        }
    }
    start[qs->n_queries] = w;
    return w;
}

/* Open-loop Poisson arrivals: n inter-arrival gaps with mean 1/rate seconds (cumulative times out). */
void synth_poisson_arrivals(uint64_t seed, uint32_t n, double rate, double *t_out) {
    rng_t r;
    rng_init(&r, seed, P_ARRIVAL, (uint64_t)(rate * 1000.0));
    double t = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        double u = rng_unif(&r);
        t += -log(1.0 - u) / rate;
        t_out[i] = t;
    }
}
