/*
 * _gen.c -- multi-threaded fills for the large seeded inputs.  Draws numbers
 * only; no sorting arithmetic.  Every value is a SplitMix64 output (Steele,
 * Lea and Flood, OOPSLA 2014) of a counter, as in sortrace_inputs/__init__.py:
 *   key(seed, tag) = mix(seed * G + tag),  draw(key, i) = mix(key + (i + 1) * G).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <unistd.h>

#define G 0x9E3779B97F4A7C15ULL

static inline uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t draw(uint64_t key, uint64_t i) { return mix(key + (i + 1) * G); }
static inline double unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

uint64_t sg_key(uint64_t seed, uint64_t tag) { return mix(seed * G + tag); }

/* ---------------------------------------------------------- thread pool */

typedef void (*range_fn)(void *ctx, size_t lo, size_t hi);
struct job { range_fn fn; void *ctx; size_t lo, hi; };
static void *run_job(void *p) { struct job *j = (struct job *)p; j->fn(j->ctx, j->lo, j->hi); return 0; }

static void parallel_for(size_t n, range_fn fn, void *ctx) {
    long nt = sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    if (nt > 64) nt = 64;
    if (n < 1 << 16) nt = 1;
    pthread_t th[64];
    struct job jobs[64];
    for (long t = 0; t < nt; t++) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * (size_t)t / (size_t)nt;
        jobs[t].hi = n * (size_t)(t + 1) / (size_t)nt;
        if (nt == 1 || pthread_create(&th[t], 0, run_job, &jobs[t]) != 0) {
            run_job(&jobs[t]);
            th[t] = 0;
        }
    }
    if (nt > 1)
        for (long t = 0; t < nt; t++) if (th[t]) pthread_join(th[t], 0);
}

/* ----------------------------------------------------------- u64 stream */

struct stream_ctx { uint64_t key, offset; uint64_t *out; };
static void stream_part(void *p, size_t lo, size_t hi) {
    struct stream_ctx *c = (struct stream_ctx *)p;
    for (size_t i = lo; i < hi; i++) c->out[i] = draw(c->key, c->offset + i);
}
void sg_stream(uint64_t key, uint64_t offset, uint64_t *out, size_t n) {
    struct stream_ctx c = {key, offset, out};
    parallel_for(n, stream_part, &c);
}

/* ------------------------------------------------------ lognormal mixture */

struct logn_ctx {
    uint64_t kc, k1, k2;
    const double *mu, *sigma, *cumw;   /* cumulative weights normalised to end at 1 */
    int ncomp;
    float *out;
};
static void logn_part(void *p, size_t lo, size_t hi) {
    struct logn_ctx *c = (struct logn_ctx *)p;
    for (size_t i = lo; i < hi; i++) {
        const double u = unit(draw(c->kc, i));
        int comp = 0;
        while (comp < c->ncomp - 1 && c->cumw[comp] <= u) comp++;
        const double u1 = unit(draw(c->k1, i)), u2 = unit(draw(c->k2, i));
        const double z = sqrt(-2.0 * log1p(-u1)) * cos(2.0 * M_PI * u2);
        c->out[i] = (float)exp(c->mu[comp] + c->sigma[comp] * z);
    }
}
void sg_lognormal(uint64_t kc, uint64_t k1, uint64_t k2, const double *mu, const double *sigma,
                  const double *cumw, int ncomp, float *out, size_t n) {
    struct logn_ctx c = {kc, k1, k2, mu, sigma, cumw, ncomp, out};
    parallel_for(n, logn_part, &c);
}

/* --------------------------------------------------- uniform + Zipf pairs */

struct zipf_ctx {
    uint64_t ku, kz;
    const double *cdf;
    size_t support;
    const uint64_t *table;
    const uint8_t *is_zipf;
    uint64_t *keys;
    uint32_t *vals;
};
static void zipf_part(void *p, size_t lo, size_t hi) {
    struct zipf_ctx *c = (struct zipf_ctx *)p;
    for (size_t i = lo; i < hi; i++) {
        if (c->is_zipf[i]) {
            const double u = unit(draw(c->kz, i));
            size_t a = 0, b = c->support;            /* first cdf entry > u */
            while (a < b) {
                const size_t m = a + (b - a) / 2;
                if (c->cdf[m] <= u) a = m + 1; else b = m;
            }
            if (a > c->support - 1) a = c->support - 1;
            c->keys[i] = c->table[a];
        } else {
            c->keys[i] = draw(c->ku, i);
        }
        c->vals[i] = (uint32_t)i;
    }
}
/* Exactly nz of the n positions get a Zipf key: selection sampling (Knuth,
 * TAOCP vol. 2, Algorithm S) picks a uniformly random subset of size nz; the
 * other positions get uniform keys.  With every key an independent draw this
 * is the concatenation of nu uniform and nz Zipf keys in uniformly random
 * order. */
void sg_zipf_pairs(uint64_t ks, uint64_t ku, uint64_t kz, const double *cdf, size_t support,
                   const uint64_t *table, size_t n, size_t nz, uint64_t *keys, uint32_t *vals,
                   uint8_t *is_zipf) {
    size_t need = nz;
    for (size_t i = 0; i < n; i++) {
        const double u = unit(draw(ks, i));
        const int take = u * (double)(n - i) < (double)need;
        is_zipf[i] = (uint8_t)take;
        need -= (size_t)take;
    }
    struct zipf_ctx c = {ku, kz, cdf, support, table, is_zipf, keys, vals};
    parallel_for(n, zipf_part, &c);
}
