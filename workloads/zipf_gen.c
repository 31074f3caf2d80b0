/*
 * Input generator for the tf-idf-like workload (no part of the method's arithmetic).
 *
 * Per set: tokens are drawn i.i.d. from Zipf(s) over ranks [0, d) (Vose's alias method) until
 * nnz distinct ranks have appeared; the set's elements are those ranks in order of first
 * appearance, and element i's weight is log(1 + count_i) * Uniform(1, 10).  Randomness:
 * xoshiro256** (Blackman and Vigna, 2018), one stream per set, seeded from four words the
 * caller draws.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

typedef struct { uint64_t s[4]; } xoshiro;

static inline uint64_t xo_next(xoshiro *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

static inline double xo_unit(xoshiro *r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

/* Vose's alias tables for weights w[0..n): prob[i] in [0, 1], alias[i]. */
int zipf_alias(int64_t n, double s, double *prob, int32_t *alias) {
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)n), *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!w || !small || !large) { free(w); free(small); free(large); return 1; }
    double tot = 0.0;
    for (int64_t i = 0; i < n; i++) { w[i] = pow((double)(i + 1), -s); tot += w[i]; }
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        w[i] = w[i] * (double)n / tot;
        if (w[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns && nl) {
        int64_t a = small[--ns], b = large[--nl];
        prob[a] = w[a];
        alias[a] = (int32_t)b;
        w[b] = (w[b] + w[a]) - 1.0;
        if (w[b] < 1.0) small[ns++] = b; else large[nl++] = b;
    }
    while (nl) { int64_t b = large[--nl]; prob[b] = 1.0; alias[b] = (int32_t)b; }
    while (ns) { int64_t a = small[--ns]; prob[a] = 1.0; alias[a] = (int32_t)a; }
    free(w); free(small); free(large);
    return 0;
}

/* Rows [s0, s1): indices/weights written at indptr[s] (indptr is the caller's CSR). */
int zipf_sets(int64_t s0, int64_t s1, const int64_t *indptr, const uint64_t *seeds, int64_t d,
              const double *prob, const int32_t *alias, uint32_t *indices, float *weights) {
    int64_t cap = 1;
    for (int64_t s = s0; s < s1; s++) {
        int64_t m = indptr[s + 1] - indptr[s];
        while (cap < 4 * m + 16) cap <<= 1;
    }
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    int32_t *val = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!key || !val || !order) { free(key); free(val); free(order); return 1; }
    for (int64_t s = s0; s < s1; s++) {
        const int64_t m = indptr[s + 1] - indptr[s];
        int64_t hc = 1;
        while (hc < 2 * m + 16) hc <<= 1;
        for (int64_t i = 0; i < hc; i++) key[i] = -1;
        xoshiro r;
        memcpy(r.s, seeds + 4 * s, 32);
        int64_t distinct = 0;
        while (distinct < m) {
            uint64_t x = xo_next(&r);
            int64_t i = (int64_t)((x >> 11) % (uint64_t)d);
            double coin = (double)(x & 0x7FF) / 2048.0 + xo_unit(&r) / 2048.0;
            if (coin >= prob[i]) i = alias[i];
            uint64_t h = (uint64_t)i * 0xD6E8FEB86659FD93ull;   /* table index only */
            int64_t slot = (int64_t)(h >> 40) & (hc - 1);
            while (key[slot] != -1 && key[slot] != i) slot = (slot + 1) & (hc - 1);
            if (key[slot] == -1) { key[slot] = i; val[slot] = 1; order[distinct++] = slot; }
            else val[slot]++;
        }
        int64_t base = indptr[s];
        for (int64_t q = 0; q < m; q++) {
            int64_t slot = order[q];
            indices[base + q] = (uint32_t)key[slot];
            weights[base + q] = (float)(log1p((double)val[slot]) * (1.0 + 9.0 * xo_unit(&r)));
        }
    }
    free(key); free(val); free(order);
    return 0;
}
