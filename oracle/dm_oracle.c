/*
 * DartMinHash ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded CPU statement of the method of
 *   T. Christiani, "DartMinHash: Fast Sketching for Weighted Sets", arXiv 2005.11547.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
 * load this file.  It shares no code, header, table or constant generator with the CUDA
 * library; the product path never calls it.
 *
 * What is computed (all comparisons in exact arithmetic on dyadic rationals):
 *
 *  Darts (Section 2, "Poisson darts"; region/area grid; Algorithm 1).  For element i and
 *  region (nu, rho), nu, rho >= 0, the region is split into 2^rho weight columns w and
 *  2^nu rank rows r.  Area (i, nu, rho, w, r) holds X ~ Poi(1) darts (Algorithm 1,
 *  "X ~ Poi(1)"); dart j < X has, with V = v/2^24, U = u/2^24 drawn from hash bits,
 *      weight = W + (w + V) * delta_nu,  W = (2^nu - 1)/t,  delta_nu = 2^nu / (t 2^rho)
 *      rank   = R + (r + U) * delta_rho, R = 2^rho - 1,     delta_rho = 2^rho / 2^nu
 *  and hits x iff weight <= x_i.  We compare t*weight <= t*x_i, which is exact because
 *  both sides are dyadic rationals.
 *
 *  Minhashes (Section 3, Theorem 1).  t = ceil(k ln k) + k; every dart is hashed to one
 *  of k buckets; minhash j is the dart of smallest rank in bucket j.  Darts are ordered
 *  by the key  (code(rank) << 32) | fp  where code() is the IEEE binary32 bit pattern of
 *  the rank rounded toward zero and fp a 32-bit hash of the dart.
 *
 *  Rank limit.  Algorithm 1 keeps darts of rank <= phi/||x||_1.  Here the limit is a
 *  binary32 value theta (any positive float near phi/||x||_1) and a dart is kept iff
 *  rank < theta, i.e. iff code(rank) < bits(theta).  Because the cut is made on the
 *  key's own rank code, a bucket that is non-empty under theta already holds its global
 *  minimum key, so the output does not depend on theta, ||x||_1 or the phi schedule.
 *
 *  Theorem 1's loop: phi = phi0, then phi <- 2 phi (or phi + 1), rerunning Algorithm 1
 *  in full, until every bucket holds a dart.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

enum { DMO_OK = 0, DMO_EINVAL = 1, DMO_ENOMEM = 2, DMO_ERANGE = 5, DMO_EOVERFLOW = 6 };

/* Region indices above this are outside the supported range (exact 64-bit device
 * arithmetic needs nu, rho <= 38). */
#define DMO_MAX_REGION 38
/* Largest phi the loop of Theorem 1 may reach before giving up. */
#define DMO_PHI_MAX 1048576.0

/* ------------------------------------------------------------------------------------ */
/* Randomness: SplitMix64's output function (Steele, Lea, Flood, OOPSLA 2014) used as a  */
/* counter-based hash.                                                                   */
/* ------------------------------------------------------------------------------------ */
#define GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define SEED_SALT  0x243F6A8885A308D3ULL
#define SLOT_SALT  0x13198A2E03707344ULL
#define BBIT_SALT  0xA4093822299F31D0ULL
#define LSH_INIT   0x082EFA98EC4E6C89ULL

static uint64_t seed_key(uint64_t seed) { return mix64(seed ^ SEED_SALT); }
static uint64_t element_key(uint64_t sigma, uint64_t i) { return mix64(sigma + GOLDEN * (i + 1)); }
static uint64_t area_key(uint64_t e, int nu, int rho, uint64_t w, uint64_t r) {
    uint64_t pack = ((uint64_t)nu << 58) | ((uint64_t)rho << 52) | (w << nu) | r;
    return mix64(e + GOLDEN * (pack + 1));
}
static uint64_t dart_key(uint64_t a, uint64_t j) { return mix64(a + GOLDEN * (j + 1)); }

/* Poisson(1) by inversion: X = number of thresholds T[n] <= u. */
static int poisson_count(uint32_t u, const uint32_t *T) {
    int x = 0;
    for (int n = 0; n < 12; n++)
        if (u >= T[n]) x++;
    return x;
}

/* ------------------------------------------------------------------------------------ */
/* Exact dyadic rationals m * 2^e (m >= 0).                                               */
/* ------------------------------------------------------------------------------------ */
typedef struct { u128 m; int e; } dy;

static int bitlen128(u128 m) {
    uint64_t hi = (uint64_t)(m >> 64), lo = (uint64_t)m;
    if (hi) return 128 - __builtin_clzll(hi);
    if (lo) return 64 - __builtin_clzll(lo);
    return 0;
}

/* -1, 0, +1 as a <, =, > b */
static int dy_cmp(dy a, dy b) {
    if (a.m == 0 || b.m == 0) return (a.m != 0) - (b.m != 0);
    int ha = bitlen128(a.m) + a.e, hb = bitlen128(b.m) + b.e;   /* a in [2^(ha-1), 2^ha) */
    if (ha != hb) return ha < hb ? -1 : 1;
    /* same magnitude: align to the smaller exponent; no overflow since top bits coincide */
    u128 am = a.m, bm = b.m;
    if (a.e > b.e) am <<= (a.e - b.e); else bm <<= (b.e - a.e);
    return (am > bm) - (am < bm);
}

static dy dy_of_float(float f) {
    uint32_t b; memcpy(&b, &f, 4);
    uint32_t ex = (b >> 23) & 0xFF, fr = b & 0x7FFFFF;
    dy r;
    if (ex == 0) { r.m = fr; r.e = -149; }
    else { r.m = fr | 0x800000u; r.e = (int)ex - 150; }
    return r;
}

/* IEEE binary32 bit pattern of the largest float <= a (round toward zero), a >= 0. */
static uint32_t rz_binary32_bits(dy a) {
    if (a.m == 0) return 0;
    int L = bitlen128(a.m);
    int X = L - 1 + a.e;                      /* floor(log2 a) */
    if (X > 127) return 0x7F7FFFFFu;
    if (X >= -126) {
        u128 mant = (L > 24) ? (a.m >> (L - 24)) : (a.m << (24 - L));
        return ((uint32_t)(X + 127) << 23) | ((uint32_t)mant & 0x7FFFFFu);
    }
    int sh = a.e + 149;
    u128 q = sh >= 0 ? (a.m << sh) : (-sh >= 128 ? 0 : (a.m >> (-sh)));
    return (uint32_t)q;
}

static u128 p2m1(int n) { return ((u128)1 << n) - 1; }          /* 2^n - 1 */

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1: DartHash_t(x, theta).  Calls `sink` for every kept dart.                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t pos;      /* position of the element inside the row */
    uint32_t i;       /* element index */
    int nu, rho;
    uint64_t w, r;
    int j;
    uint32_t u, v;    /* 24-bit uniforms */
    uint32_t code;    /* rank code */
    uint64_t q;       /* bucket/fingerprint hash */
} dmo_dart;

typedef void (*dart_sink)(void *ctx, const dmo_dart *d);

typedef struct { int64_t areas, darts, kept; } dmo_work;

/* Algorithm 1.  scale: every weight counts as x_i 2^scale (the exact power-of-two normalisation
   of a weight class, Section 3); 0 for the plain method. */
static int darthash_s(const uint32_t *idx, const float *wt, int64_t nnz, int64_t t, uint64_t sigma,
                      const uint32_t *T, float theta, int scale, dart_sink sink, void *ctx, dmo_work *work) {
    dy th = dy_of_float(theta);
    for (int64_t p = 0; p < nnz; p++) {
        float xi = wt[p];
        if (!(xi > 0.0f)) continue;                               /* i in {j | x_j > 0} */
        dy xf = dy_of_float(xi);
        xf.e += scale;                                            /* x_i 2^scale, exact */
        dy y = { (u128)t * xf.m, xf.e };                          /* t * x_i, exact */
        uint64_t e = element_key(sigma, idx[p]);
        /* nu = 0 .. floor(log2(1 + t x_i)):  continue while 2^nu - 1 <= t x_i */
        for (int nu = 0; ; nu++) {
            dy wlo = { p2m1(nu), 0 };
            if (dy_cmp(wlo, y) > 0) break;
            if (nu > DMO_MAX_REGION) return DMO_ERANGE;
            /* rho = 0 .. : continue while R = 2^rho - 1 < theta */
            for (int rho = 0; ; rho++) {
                dy rlo = { p2m1(rho), 0 };
                if (dy_cmp(rlo, th) >= 0) break;
                if (rho > DMO_MAX_REGION || nu + rho > 52) return DMO_ERANGE;
                for (uint64_t w = 0; w < ((uint64_t)1 << rho); w++) {
                    /* break if x_i < W + w delta_nu; scaled by t 2^rho:
                       (2^nu - 1) 2^rho + w 2^nu  vs  t x_i 2^rho */
                    dy cw = { (p2m1(nu) << rho) + ((u128)w << nu), -rho };
                    if (dy_cmp(y, cw) < 0) break;
                    for (uint64_t r = 0; r < ((uint64_t)1 << nu); r++) {
                        /* break if theta <= R + r delta_rho; scaled by 2^nu:
                           (2^rho - 1) 2^nu + r 2^rho */
                        dy cr = { (p2m1(rho) << nu) + ((u128)r << rho), -nu };
                        if (dy_cmp(th, cr) <= 0) break;
                        uint64_t a = area_key(e, nu, rho, w, r);
                        int X = poisson_count((uint32_t)(a >> 32), T);
                        if (work) work->areas++;
                        for (int j = 0; j < X; j++) {
                            uint64_t d = dart_key(a, (uint64_t)j);
                            uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & 0xFFFFFFu;
                            if (work) work->darts++;
                            /* t * weight = 2^nu - 1 + (w + V) 2^(nu-rho), times 2^(rho+24) */
                            dy sw = { (p2m1(nu) << (rho + 24)) + ((((u128)w << 24) | v) << nu), -rho - 24 };
                            /* rank = 2^rho - 1 + (r + U) 2^(rho-nu), times 2^(nu+24) */
                            dy sr = { (p2m1(rho) << (nu + 24)) + ((((u128)r << 24) | u) << rho), -nu - 24 };
                            if (dy_cmp(sw, y) > 0) continue;                /* weight <= x_i */
                            if (dy_cmp(sr, th) >= 0) continue;              /* rank < theta */
                            if (work) work->kept++;
                            dmo_dart D;
                            D.pos = p; D.i = idx[p]; D.nu = nu; D.rho = rho; D.w = w; D.r = r; D.j = j;
                            D.u = u; D.v = v;
                            D.code = rz_binary32_bits(sr);
                            D.q = mix64(d ^ SLOT_SALT);
                            sink(ctx, &D);
                        }
                    }
                }
            }
        }
    }
    return DMO_OK;
}

static int darthash(const uint32_t *idx, const float *wt, int64_t nnz, int64_t t, uint64_t sigma,
                    const uint32_t *T, float theta, dart_sink sink, void *ctx, dmo_work *work) {
    return darthash_s(idx, wt, nnz, t, sigma, T, theta, 0, sink, ctx, work);
}

static uint32_t fastrange32(uint32_t h, uint32_t n) { return (uint32_t)(((uint64_t)h * n) >> 32); }
static uint64_t dart_minkey(const dmo_dart *d) { return ((uint64_t)d->code << 32) | (uint32_t)d->q; }

/* ------------------------------------------------------------------------------------ */
/* Theorem 1: k independent minhashes.                                                   */
/* ------------------------------------------------------------------------------------ */
typedef struct { uint64_t *slots; int32_t k; } sketch_ctx;

static void sketch_sink(void *c, const dmo_dart *d) {
    sketch_ctx *s = (sketch_ctx *)c;
    uint32_t j = fastrange32((uint32_t)(d->q >> 32), (uint32_t)s->k);
    uint64_t key = dart_minkey(d);
    if (key < s->slots[j]) s->slots[j] = key;
}

static int check_row(const float *wt, int64_t nnz, double *l1) {
    double s = 0.0;
    for (int64_t p = 0; p < nnz; p++) {
        float x = wt[p];
        if (!(x >= 0.0f) || isinf(x)) return DMO_EINVAL;          /* NaN, negative, inf */
        s += (double)x;
    }
    *l1 = s;
    return DMO_OK;
}

/* One set: loop over phi as in Theorem 1. schedule 0: phi <- 2 phi, 1: phi <- phi + 1. */
static int sketch_one(const uint32_t *idx, const float *wt, int64_t nnz, int32_t k, uint64_t sigma,
                      int64_t t, const uint32_t *T, double phi0, int32_t schedule,
                      uint64_t *out, int64_t *work4) {
    double l1;
    int rc = check_row(wt, nnz, &l1);
    for (int32_t j = 0; j < k; j++) out[j] = UINT64_MAX;
    if (rc) return rc;
    dmo_work W = {0, 0, 0};
    int64_t passes = 0;
    if (l1 > 0.0) {
        for (double phi = phi0; ; phi = schedule == 0 ? 2.0 * phi : phi + 1.0) {
            if (phi > DMO_PHI_MAX) return DMO_EOVERFLOW;
            float theta = (float)(phi / l1);
            if (!(theta > 0.0f) || isinf(theta)) return DMO_ERANGE;
            for (int32_t j = 0; j < k; j++) out[j] = UINT64_MAX;
            sketch_ctx c = { out, k };
            rc = darthash(idx, wt, nnz, t, sigma, T, theta, sketch_sink, &c, &W);
            passes++;
            if (rc) return rc;
            int full = 1;
            for (int32_t j = 0; j < k; j++) full &= (out[j] != UINT64_MAX);
            if (full) break;
        }
    }
    if (work4) { work4[0] = W.areas; work4[1] = W.darts; work4[2] = W.kept; work4[3] = passes; }
    return DMO_OK;
}

int dmo_sketch(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n_sets,
               int32_t k, uint64_t seed, int64_t t, const uint32_t *T, double phi0, int32_t schedule,
               uint64_t *out, int64_t *work) {
    if (k < 1 || t < 1 || !(phi0 > 0.0)) return DMO_EINVAL;
    uint64_t sigma = seed_key(seed);
    int status = DMO_OK;
    for (int64_t s = 0; s < n_sets; s++) {
        int64_t b = indptr[s], e = indptr[s + 1];
        int rc = sketch_one(indices + b, weights + b, e - b, k, sigma, t, T, phi0, schedule,
                            out + s * (int64_t)k, work ? work + 4 * s : NULL);
        if (rc && !status) status = rc;
    }
    return status;
}

/* b-bit minhash (Section 1.1, "Similarity estimation"): each minhash is mapped by a random
 * hash to b bits; slot j occupies bits (j b) mod 64 of word floor(j b / 64), LSB first;
 * a row has ceil(k b / 64) words and unused high bits of the last word are zero. */
int dmo_sketch_bbit(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n_sets,
                    int32_t k, int32_t b, uint64_t seed, int64_t t, const uint32_t *T,
                    uint64_t *out_words, uint64_t *out_keys) {
    if (!(b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32)) return DMO_EINVAL;
    if (k < 1) return DMO_EINVAL;
    int64_t words = ((int64_t)k * b + 63) / 64;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)k);
    if (!keys) return DMO_ENOMEM;
    uint64_t sigma = seed_key(seed);
    int status = DMO_OK;
    uint64_t mask = (1ULL << b) - 1;
    for (int64_t s = 0; s < n_sets; s++) {
        int64_t bgn = indptr[s], end = indptr[s + 1];
        int rc = sketch_one(indices + bgn, weights + bgn, end - bgn, k, sigma, t, T, 1.0, 0, keys, NULL);
        if (rc && !status) status = rc;
        uint64_t *ow = out_words + s * words;
        for (int64_t q = 0; q < words; q++) ow[q] = 0;
        for (int32_t j = 0; j < k; j++) {
            uint64_t beta = mix64(keys[j] ^ BBIT_SALT) & mask;
            int64_t bit = (int64_t)j * b;
            ow[bit / 64] |= beta << (bit % 64);
        }
        if (out_keys) memcpy(out_keys + s * (int64_t)k, keys, sizeof(uint64_t) * (size_t)k);
    }
    free(keys);
    return status;
}

/* ------------------------------------------------------------------------------------ */
/* (L, K) LSH (Section 3, "Bottom-k minhash and fast approximate near neighbor search"):  */
/* t = L K, darts hashed to L buckets, bucket l's value is a hash of its K smallest keys  */
/* in increasing order.  phi doubles until every bucket holds at least K darts.          */
/* ------------------------------------------------------------------------------------ */
typedef struct { uint64_t *key; uint32_t *bucket; int64_t n, cap; int32_t L; int oom; } lsh_ctx;

static void lsh_sink(void *c, const dmo_dart *d) {
    lsh_ctx *s = (lsh_ctx *)c;
    if (s->n == s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 1024;
        uint64_t *nk = (uint64_t *)realloc(s->key, sizeof(uint64_t) * (size_t)nc);
        if (nk) s->key = nk;
        uint32_t *nb = (uint32_t *)realloc(s->bucket, sizeof(uint32_t) * (size_t)nc);
        if (nb) s->bucket = nb;
        if (!nk || !nb) { s->oom = 1; return; }
        s->cap = nc;
    }
    s->key[s->n] = dart_minkey(d);
    s->bucket[s->n] = fastrange32((uint32_t)(d->q >> 32), (uint32_t)s->L);
    s->n++;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* (L, K) LSH; scale (may be NULL): set s's weights count as x_i 2^scale[s] (weight classes
   normalised to ||x||_1 in [1, 2), Section 3). */
int dmo_lsh_scaled(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n_sets,
                   int32_t L, int32_t K, uint64_t seed, const uint32_t *T, double phi0, const int32_t *scale,
                   uint32_t *out, int64_t *work) {
    if (L < 1 || K < 1) return DMO_EINVAL;
    int64_t t = (int64_t)L * K;
    uint64_t sigma = seed_key(seed);
    int status = DMO_OK;
    lsh_ctx c = { NULL, NULL, 0, 0, L, 0 };
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * 1024);
    int64_t tmpcap = 1024;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    if (!tmp || !cnt) { free(tmp); free(cnt); return DMO_ENOMEM; }
    for (int64_t s = 0; s < n_sets; s++) {
        int64_t bgn = indptr[s], end = indptr[s + 1];
        const uint32_t *idx = indices + bgn; const float *wt = weights + bgn; int64_t nnz = end - bgn;
        uint32_t *o = out + s * (int64_t)L;
        for (int32_t l = 0; l < L; l++) o[l] = UINT32_MAX;
        double l1;
        int rc = check_row(wt, nnz, &l1);
        dmo_work W = {0, 0, 0};
        int64_t passes = 0;
        if (!rc && l1 > 0.0) {
            const int sc = scale ? scale[s] : 0;
            for (double phi = phi0; ; phi *= 2.0) {
                if (phi > DMO_PHI_MAX) { rc = DMO_EOVERFLOW; break; }
                float theta = (float)(phi / ldexp(l1, sc));
                if (!(theta > 0.0f) || isinf(theta)) { rc = DMO_ERANGE; break; }
                c.n = 0;
                rc = darthash_s(idx, wt, nnz, t, sigma, T, theta, sc, lsh_sink, &c, &W);
                passes++;
                if (c.oom) rc = DMO_ENOMEM;
                if (rc) break;
                for (int32_t l = 0; l < L; l++) cnt[l] = 0;
                for (int64_t q = 0; q < c.n; q++) cnt[c.bucket[q]]++;
                int full = 1;
                for (int32_t l = 0; l < L; l++) full &= (cnt[l] >= K);
                if (!full) continue;
                for (int32_t l = 0; l < L; l++) {
                    if (cnt[l] > tmpcap) {
                        uint64_t *nt = (uint64_t *)realloc(tmp, sizeof(uint64_t) * (size_t)cnt[l]);
                        if (!nt) { rc = DMO_ENOMEM; break; }
                        tmp = nt; tmpcap = cnt[l];
                    }
                    int64_t m = 0;
                    for (int64_t q = 0; q < c.n; q++) if (c.bucket[q] == (uint32_t)l) tmp[m++] = c.key[q];
                    qsort(tmp, (size_t)m, sizeof(uint64_t), cmp_u64);
                    uint64_t h = LSH_INIT;
                    for (int32_t q = 0; q < K; q++) h = mix64(h ^ tmp[q]);
                    o[l] = (uint32_t)(h >> 32);
                }
                break;
            }
        }
        if (rc && !status) status = rc;
        if (work) { work[4 * s] = W.areas; work[4 * s + 1] = W.darts; work[4 * s + 2] = W.kept; work[4 * s + 3] = passes; }
    }
    free(c.key); free(c.bucket); free(tmp); free(cnt);
    return status;
}

int dmo_lsh(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n_sets,
            int32_t L, int32_t K, uint64_t seed, const uint32_t *T, double phi0,
            uint32_t *out, int64_t *work) {
    return dmo_lsh_scaled(indptr, indices, weights, n_sets, L, K, seed, T, phi0, NULL, out, work);
}

/* ------------------------------------------------------------------------------------ */
/* Bottom-k weighted sketch (Section 3, "Bottom-k minhash"): t = k; phi is raised until   */
/* DartHash returns at least k darts; the k smallest keys in increasing order.            */
/* ------------------------------------------------------------------------------------ */
int dmo_bottomk(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n_sets,
                int32_t k, uint64_t seed, const uint32_t *T, double phi0, uint64_t *out, int64_t *work) {
    if (k < 1) return DMO_EINVAL;
    uint64_t sigma = seed_key(seed);
    int status = DMO_OK;
    lsh_ctx c = { NULL, NULL, 0, 0, 1, 0 };
    for (int64_t s = 0; s < n_sets; s++) {
        int64_t bgn = indptr[s], end = indptr[s + 1];
        const uint32_t *idx = indices + bgn; const float *wt = weights + bgn; int64_t nnz = end - bgn;
        uint64_t *o = out + s * (int64_t)k;
        for (int32_t j = 0; j < k; j++) o[j] = UINT64_MAX;
        double l1;
        int rc = check_row(wt, nnz, &l1);
        dmo_work W = {0, 0, 0};
        int64_t passes = 0;
        if (!rc && l1 > 0.0) {
            for (double phi = phi0; ; phi *= 2.0) {
                if (phi > DMO_PHI_MAX) { rc = DMO_EOVERFLOW; break; }
                float theta = (float)(phi / l1);
                if (!(theta > 0.0f) || isinf(theta)) { rc = DMO_ERANGE; break; }
                c.n = 0;
                rc = darthash(idx, wt, nnz, (int64_t)k, sigma, T, theta, lsh_sink, &c, &W);
                passes++;
                if (c.oom) rc = DMO_ENOMEM;
                if (rc) break;
                if (c.n < k) continue;
                qsort(c.key, (size_t)c.n, sizeof(uint64_t), cmp_u64);
                for (int32_t j = 0; j < k; j++) o[j] = c.key[j];
                break;
            }
        }
        if (rc && !status) status = rc;
        if (work) { work[4 * s] = W.areas; work[4 * s + 1] = W.darts; work[4 * s + 2] = W.kept; work[4 * s + 3] = passes; }
    }
    free(c.key); free(c.bucket);
    return status;
}

/* ------------------------------------------------------------------------------------ */
/* Test access: the kept darts of one row at a fixed theta (Algorithm 1's output set D).  */
/* ------------------------------------------------------------------------------------ */
typedef struct { dmo_dart *buf; int64_t n, cap; } collect_ctx;

static void collect_sink(void *c, const dmo_dart *d) {
    collect_ctx *s = (collect_ctx *)c;
    if (s->n < s->cap) s->buf[s->n] = *d;
    s->n++;
}

/* Returns the number of kept darts (may exceed cap; only cap are stored), or -(error). */
int64_t dmo_darthash(const uint32_t *idx, const float *wt, int64_t nnz, int64_t t, uint64_t seed,
                     const uint32_t *T, float theta, dmo_dart *out, int64_t cap, int64_t *work3) {
    double l1;
    int rc = check_row(wt, nnz, &l1);
    if (rc) return -rc;
    collect_ctx c = { out, 0, cap };
    dmo_work W = {0, 0, 0};
    rc = darthash(idx, wt, nnz, t, seed_key(seed), T, theta, collect_sink, &c, &W);
    if (rc) return -rc;
    if (work3) { work3[0] = W.areas; work3[1] = W.darts; work3[2] = W.kept; }
    return c.n;
}

int64_t dmo_dart_record_size(void) { return (int64_t)sizeof(dmo_dart); }

uint64_t dmo_mix64(uint64_t z) { return mix64(z); }
