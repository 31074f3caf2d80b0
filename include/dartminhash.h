/*
 * dartminhash.h -- C ABI of the GB300 (sm_103a) DartMinHash library, libdartminhash.so.
 *
 * Method: T. Christiani, "DartMinHash: Fast Sketching for Weighted Sets" (arXiv 2005.11547).
 *   DartHash (Section 2, Algorithm 1) enumerates the darts of a hashed Poisson dart process
 *   that hit a weighted set x with rank below a limit; DartMinHash (Section 3, Theorem 1)
 *   hashes every dart to one of k buckets and keeps the smallest-rank dart per bucket,
 *   repeating with a doubled limit while a bucket is empty.
 *
 * Conventions shared by every call
 *   - Sets come as CSR: indptr int64[n_sets + 1] (indptr[0] = 0, non-decreasing), indices
 *     uint32[indptr[n_sets]] (element ids i), weights float32[indptr[n_sets]] (x_i).
 *     Weights must be finite and >= 0 (the domain R^d_{>=0} of Section 1); zero weights are
 *     skipped (Algorithm 1 visits only {i | x_i > 0}); element order inside a row does not
 *     matter.  A repeated index acts as the largest of its weights for dm_sketch and
 *     dm_sketch_bbit (a minimum ignores repeated darts); for dm_lsh it contributes its darts once
 *     per occurrence, so rows passed to dm_lsh should not repeat an index.
 *   - Unless a call says otherwise, every array argument is a DEVICE pointer owned by the
 *     caller; the library reads/writes it only on `stream` and keeps no reference after the
 *     work queued on `stream` completes.  `stream` is a cudaStream_t passed as void* (NULL =
 *     the legacy default stream).  indptr, indices and weights must be aligned to their
 *     element size (8, 4 and 4 bytes); a misaligned one is refused with DM_EINVAL before any
 *     launch.
 *   - Output key layout: out[s * k + j] is minhash j of set s, the 64-bit key
 *         (code(rank) << 32) | fingerprint
 *     where code(rank) is the IEEE binary32 bit pattern of the winning dart's rank rounded
 *     toward zero and fingerprint a 32-bit hash of the dart.  Keys of two sets are equal iff
 *     the same dart wins (up to a 2^-32 fingerprint coincidence at equal rank codes).  A set
 *     with no positive weight gets 0xFFFFFFFFFFFFFFFF in every slot.
 *   - The same (row, k, seed) always gives the same bits on every GPU, batch composition,
 *     launch form and tuning choice.
 *   - Return value: DM_OK or an error code.  Argument errors found on the host are returned
 *     at once and nothing is queued.  Errors found by the kernels (a negative/NaN/Inf weight:
 *     DM_EINVAL; a weight with t*x_i >= 2^39 - 1 or a set needing a rank limit >= 2^39 - 1:
 *     DM_ERANGE) are recorded in the context and returned by dm_sync_status(); the rows they
 *     concern are filled with 0xFF bytes.
 *   - Thread safety: one dm_ctx per host thread (or serialize calls on a context).
 */
#ifndef DARTMINHASH_H
#define DARTMINHASH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dm_ctx dm_ctx;

enum dm_status {
    DM_OK = 0,
    DM_EINVAL = 1,     /* invalid argument or invalid weight */
    DM_ENOMEM = 2,     /* device or pinned allocation failed, or over the memory budget */
    DM_ECUDA = 3,      /* a CUDA runtime call failed */
    DM_ETIMEOUT = 4,   /* a bounded device wait gave up */
    DM_ERANGE = 5,     /* input outside the supported numeric range (see above) */
    DM_EOVERFLOW = 6,  /* the doubling loop of Theorem 1 reached its limit */
    DM_EAGAIN = 7,     /* dm_server_submit: the admission budget is full now; retry later */
    DM_ECHECK = 8      /* checked build only (dm_build_flags() & 1): an internal index check
                          failed, a defect of the library; the access it guarded was skipped */
};

/* Create a context on CUDA device `device`.  `mem_budget_bytes` caps the device scratch the
 * context may allocate (0 = no cap).  Uploads the Poisson(1) inversion table of
 * Algorithm 1 to the device.  *out receives the context (owned by the caller; release with
 * dm_destroy).  Returns DM_EINVAL for a bad device, DM_ECUDA on a runtime failure. */
int dm_create(dm_ctx **out, int device, size_t mem_budget_bytes);

/* Release the context and everything it allocated.  NULL is accepted. */
int dm_destroy(dm_ctx *ctx);

/* k independent weighted minhashes per set (Theorem 1, with Algorithm 1 as the inner
 * step; t = ceil(k ln k) + k).  out: uint64[n_sets * k] (layout above).  1 <= k <= 8192,
 * n_sets >= 0; seed selects the hash functions. */
int dm_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
              int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream);

/* b-bit minhash (Section 1.1, "Similarity estimation": each minhash mapped by a random hash to
 * b bits; for b = 1, 64 minhashes per machine word).  b in {1, 2, 4, 8, 16, 32}.
 * out_words: uint64[n_sets * W], W = ceil(k * b / 64); slot j of set s occupies bits
 * (j*b) mod 64 .. +b-1 of word s*W + floor(j*b/64), least significant bit first; unused high
 * bits of a row's last word are zero.  The b-bit value of a slot is the low b bits of
 * SplitMix64's output function applied to (key XOR 0xA4093822299F31D0).  out_keys, when not
 * NULL, also receives the uint64 keys exactly as dm_sketch writes them (uint64[n_sets * k]). */
int dm_sketch_bbit(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                   int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words,
                   uint64_t *out_keys, void *stream);

/* Fully independent (L, K) LSH values (Section 1.2 "Fast similarity search" and Section 3,
 * "Bottom-k minhash and fast approximate near neighbor search"): t = L*K, darts hashed to
 * L buckets, the rank limit doubled until every bucket holds >= K darts; table l's value is
 * the high 32 bits of the chain h <- SplitMix64out(h XOR key_m) over the bucket's K smallest
 * keys in increasing order, from h = 0x082EFA98EC4E6C89.  Two sets collide in a table with
 * probability J^K, independently across tables.  out: uint32[n_sets * L] (row-major); a set
 * with no positive weight gets 0xFFFFFFFF.  1 <= L <= 1024, 1 <= K <= 32, and a set's bucket
 * state (8 L K + 4 L bytes, plus about 4.9 KB of walk tables and queues per warp) must fit in
 * shared memory, else DM_EINVAL. */
int dm_lsh(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
           int64_t n_sets, int32_t L, int32_t K, uint64_t seed, uint32_t *out, void *stream);

/* dm_lsh on weight-class-normalised data (Section 3: split the data into classes
 * ||x||_1 in [2^c, 2^(c+1)) and normalise each class to ||x||_1 in [1, 2), which bounds the work of
 * sets with very large or very small norms).  scale_exp: device int32[n_sets]; set s's weights
 * count as x_i 2^scale_exp[s], exactly (the scaling acts on the exponent, so no weight is rounded).
 * Normalising class c means scale_exp = -c; a query probes a neighbouring class c' by hashing with
 * -c'.  The same (row, scale) always gives the same values; scale 0 equals dm_lsh. */
int dm_lsh_scaled(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                  int64_t n_sets, int32_t L, int32_t K, uint64_t seed, const int32_t *scale_exp, uint32_t *out,
                  void *stream);

/* Weight class of each set (Section 3, "Bottom-k minhash and fast approximate near neighbor
 * search"): out[s] = floor(log2 ||x||_1), where ||x||_1 is the exact sum of the set's positive
 * finite weights (an integer sum of their significands, so a norm next to a power of two always
 * lands in the right class, whatever the element order); zero, negative, NaN and infinite weights
 * take no part, and a set without a positive finite weight gets 0.  Classes run from -149 to
 * 128 + log2(nnz); rows must have fewer than 2^32 elements.  Device int32 out[n_sets] (may be
 * NULL); scale_out (may be NULL) receives norm_exp - out[s], the scale for dm_lsh_scaled that puts the class's norms in
 * [2^norm_exp, 2^(norm_exp+1)) (Section 3 normalises to [1, 2), norm_exp = 0; a larger range keeps
 * the first rank limit phi0 / ||x||_1 below 1, where the enumeration is cheapest). */
int dm_weight_classes(dm_ctx *ctx, const int64_t *indptr, const float *weights, int64_t n_sets, int32_t *out,
                      int32_t *scale_out, int32_t norm_exp, void *stream);

/* Bottom-k weighted sketch (Section 3, "Bottom-k minhash and fast approximate near neighbor
 * search": with t = k, raise phi until DartHash returns at least k darts and keep them sorted by
 * rank).  out: uint64[n_sets * k]; row s holds the k smallest keys of set s's darts (the same
 * 64-bit keys as dm_sketch: rank code << 32 | fingerprint, the fingerprint being the low 32 bits
 * of the bucket hash) in increasing order.  A set with no positive weight gets all ones.  The
 * union estimator |S_k(x v y) n S_k(x) n S_k(y)| / k of the weighted Jaccard similarity, with
 * x v y the coordinatewise maximum, is Bin(k, J) / k.  1 <= k <= 1024 (the candidate buffer,
 * 8 * 2^ceil(log2(max(2k, k + 32))) bytes per set, lives in shared memory). */
int dm_bottomk(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
               int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream);

/* LSH tables for approximate near neighbor search (Section 1.2, "Fast similarity search", and
 * Section 3): L hash tables keyed by the L values dm_lsh / dm_lsh_scaled give each point.  A query
 * gets every point that shares a value with it in at least one table (for a point at weighted
 * Jaccard similarity J, with probability 1 - (1 - J^K)^L).  The index lives on `device` and holds
 * up to `capacity` points (capacity * L <= 2^31 - 1; about 24 L bytes per point of capacity).
 *   create: empty index.  insert: n points, values uint32[n * L] (row-major, device), ids int64[n]
 *   (device; NULL = consecutive ids from the number of points already inserted); DM_ENOMEM past
 *   the capacity.  query: m queries, values uint32[m * L]; counts int32[m] receives the number of
 *   distinct candidates (-1 if a query gathers more than 2,048 (point, table) collisions), out_ids
 *   int64[m * max_candidates] the smallest max_candidates candidate ids in increasing order, padded
 *   with -1 (1 <= max_candidates <= 2,048).  All asynchronous on `stream`; status returns (and
 *   clears) an insertion error recorded by the device (DM_EOVERFLOW: a table probe gave up). */
typedef struct dm_lsh_index dm_lsh_index;
int dm_lsh_index_create(dm_lsh_index **out, int device, int32_t L, int64_t capacity);
int dm_lsh_index_insert(dm_lsh_index *ix, const uint32_t *values, const int64_t *ids, int64_t n, void *stream);
int dm_lsh_index_query(dm_lsh_index *ix, const uint32_t *queries, int64_t m, int32_t max_candidates,
                       int32_t *counts, int64_t *out_ids, void *stream);
int dm_lsh_index_size(dm_lsh_index *ix, int64_t *n);
int dm_lsh_index_status(dm_lsh_index *ix, void *stream);
int dm_lsh_index_destroy(dm_lsh_index *ix);

/* Similarity counts of sketches (Section 1.1, "Similarity estimation"): for each pair of rows,
 * the number m of the k slots whose values agree.  bits = 0: rows of k uint64 keys from dm_sketch
 * (E[m] = k J, Eq. 1, so m / k estimates the weighted Jaccard similarity J); bits = b in
 * {1, 2, 4, 8, 16, 32}: rows of W = ceil(k b / 64) packed words from dm_sketch_bbit
 * (E[m] = k (J + (1 - J) 2^-b), so J is estimated by (m / k - 2^-b) / (1 - 2^-b)).  Both batches
 * must come from the same k, b and seed.  mode 0 (pairs): n_a == n_c, out[i] compares row i of a
 * with row i of c (uint32[n_a]); mode 1 (cross): out[i * n_c + j] compares row i of a with row j
 * of c (uint32[n_a * n_c]; n_a <= 2,097,120, and W <= 64 for b-bit rows).  Device pointers,
 * asynchronous on `stream`. */
int dm_compare(dm_ctx *ctx, const uint64_t *a, const uint64_t *c, int64_t n_a, int64_t n_c, int32_t k,
               int32_t bits, int32_t mode, uint32_t *out, void *stream);

/* Weighted Jaccard estimates from the counts of dm_compare (Section 1.1, "Similarity
 * estimation"): out[i] = m[i] / k for keys (bits = 0; Eq. 1 makes it unbiased), and
 * (m[i] / k - 2^-b) / (1 - 2^-b) for b-bit fields (bits = b), each step a correctly rounded
 * binary64 operation in that order.  matches: device uint32[n]; out: device double[n].  Needs no
 * context; runs on the current device, asynchronously on `stream`. */
int dm_estimate_jaccard(const uint32_t *matches, int64_t n, int32_t k, int32_t bits, double *out, void *stream);

/* Top-k neighbours by estimated similarity (Section 1.1, "Similarity estimation": the agreeing
 * slots m of two sketches estimate their weighted Jaccard similarity, so the rows of c with the
 * largest m are the most similar): for each row i of a, the `topk` rows j of c with the largest
 * dm_compare count m(i, j), in decreasing order of m, rows with equal m in increasing order of j.
 * Rows as for dm_compare (bits = 0: k uint64 keys; bits = b: W = ceil(k b / 64) words of b-bit
 * fields, W <= 64), from the same k, b and seed.  out_idx, out_count: device uint32[n_a * topk];
 * entry i * topk + t is the t-th neighbour of row i and its count; when n_c < topk the entries
 * past n_c are 0xFFFFFFFF with count 0.  1 <= topk <= 32, n_c < 2^31.  Asynchronous on `stream`
 * (scratch of 8 n_a topk bytes per span of c rows is allocated stream-ordered when the search
 * splits c into spans). */
int dm_compare_topk(dm_ctx *ctx, const uint64_t *a, const uint64_t *c, int64_t n_a, int64_t n_c, int32_t k,
                    int32_t bits, int32_t topk, uint32_t *out_idx, uint32_t *out_count, void *stream);

/* Wide-range minhash keys: 64-bit element ids and binary64 weights, for the norms the binary32
 * entry points cannot reach (Section 4, "Synthetic data", hashes 64-bit ids with double weights;
 * Table 1 runs ||x||_1 = 2^{+-64} and 2^{+-512}).  Same dart process as dm_sketch (Section 2,
 * Algorithm 1, Theorem 1), with keys of their own (so they never compare with dm_sketch's):
 *   - area (nu, rho, w, r) of element i is hashed in two levels, region key
 *     z = M(e_i + gamma (1 + 2^16 nu + rho)) and area key a = M(z + gamma (1 + 2^32 w + r));
 *   - a key is (code << 32) | (q mod 2^32), where code is the upper 32 bits of the binary64 pattern
 *     of the dart's rank rounded toward zero (sign, 11 exponent and 20 fraction bits).
 * indptr int64[n_sets + 1], indices uint64[nnz], weights float64[nnz]: device arrays, CSR as for
 * dm_sketch; out: uint64[n_sets * k] device array.  1 <= k <= 1024.  Asynchronous on `stream`.
 * Errors recorded for dm_sync_status (the set's row then holds all ones): DM_EINVAL for a
 * negative, NaN or infinite weight; DM_ERANGE for a weight >= 2^960 or a set whose largest weight
 * is positive and below 2^-990 (both keep every rank and limit a normal binary64 number);
 * DM_EOVERFLOW after 17 passes of the doubling loop.  A set without a positive weight gets all
 * ones.  DM_OPT_COUNTERS, when set, accumulates areas, darts, kept darts and passes. */
int dm_sketch_f64(dm_ctx *ctx, const int64_t *indptr, const uint64_t *indices, const double *weights,
                  int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream);

/* b-bit sketches of the wide-range keys: the words dm_sketch_bbit would write for these keys
 * (b in {1, 2, 4, 8, 16, 32}; out_words uint64[n_sets * ceil(k b / 64)], same layout).  b = 0
 * writes keys only.  out_keys (may be NULL when b > 0) receives the keys of dm_sketch_f64.  The
 * rows of sets with an error hold 0xFF bytes, in both outputs. */
int dm_sketch_f64_bbit(dm_ctx *ctx, const int64_t *indptr, const uint64_t *indices, const double *weights,
                       int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words, uint64_t *out_keys,
                       void *stream);

/* Measurement helper (no paper counterpart): the integer-issue ceiling of the counter-based hash.
 * Launches `blocks` blocks of 256 threads; each thread applies SplitMix64's output function
 * 4 * iters times (four independent chains) and writes the xor of its chains to out[thread]
 * (device uint64[blocks * 256]).  Asynchronous on `stream`: time it with events on that stream.
 * 4 * iters * 256 * blocks mixes, 18 int32 operations each, against SMs x 128 lanes x clock. */
int dm_mix64_burn(int64_t blocks, int32_t iters, uint64_t seed, uint64_t *out, void *stream);

/* dm_sketch / dm_sketch_bbit with HOST arrays: indptr, indices, weights, out_keys and
 * out_words are host pointers (page-locked memory gives full speed).  b = 0 computes keys
 * only (out_keys required, out_words ignored); b in {1, 2, 4, 8, 16, 32} also writes the b-bit
 * words (out_keys may then be NULL).  Two ways to move the data (DM_OPT_HOST_MODE): in place,
 * where the kernels read the page-locked, mapped host arrays and write the outputs there
 * directly (no device copy of the batch is made); or staged, where the library copies the batch
 * to context-owned device buffers on `stream` in chunks, overlapping the copies of one chunk with
 * the kernel of the previous one.  Either way the call returns after every output is in host
 * memory (synchronous).  Returns DM_ENOMEM if the staging buffers would exceed the context's
 * memory budget. */
int dm_sketch_host(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                   int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_keys,
                   uint64_t *out_words, void *stream);

/* Largest n_sets that dm_sketch_noalloc accepts. */
#define DM_NOALLOC_MAX_SETS 262144

/* dm_sketch without a context and without any device allocation.  (The paper has no
 * counterpart: this exists for host programs that do not allow a library to allocate, such as a
 * framework that hands all device memory to its own caching allocator, or a process that
 * reserved the whole device.)  Same arguments, outputs and bits as dm_sketch, with the library's
 * default phi0 (1.25) and automatic launch shape, on the current CUDA device; every pointer must
 * be memory of that device.  The library's scratch for this call (work queue, counters, status)
 * is a fixed device array of about 1 MiB that every GPU loading the library holds until the
 * process exits; n_sets above DM_NOALLOC_MAX_SETS is rejected with DM_EINVAL before any GPU
 * work.  All calls share that array, so calls whose work overlaps on a GPU (other streams or
 * host threads) race and may return wrong keys.  The first call on a device performs a one-time
 * set-up (finding the array's device address, loading the Poisson table, raising the kernels'
 * shared-memory limit); a set-up that fails is tried again by the next call.  The call is
 * synchronous: it waits for `stream` and returns the first error the kernels recorded
 * (DM_EINVAL for a bad weight, DM_ERANGE ...).  It therefore cannot be recorded into a CUDA
 * graph: on a stream that is being captured it returns DM_EINVAL without doing anything. */
int dm_sketch_noalloc(const int64_t *indptr, const uint32_t *indices, const float *weights,
                      int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream);

/* Wait for `stream`, then return (and clear) the first error recorded by a kernel of this
 * context, or DM_ECUDA if the stream itself failed. */
int dm_sync_status(dm_ctx *ctx, void *stream);

/* Static English description of a status code. */
const char *dm_strerror(int status);

/* Build flags of the loaded library: bit 0 set = the checked build (libdartminhash_checked.so,
 * compiled with -DDM_CHECKED): every kernel also checks its shared-memory ring, table and bucket
 * indices, records the first failed check instead of making the access, and dm_sync_status then
 * returns DM_ECHECK.  The product build (bit 0 clear) has no such checks. */
int32_t dm_build_flags(void);

/* Tuning and instrumentation options (dm_set_option).  None of them changes any output bit. */
enum dm_option {
    DM_OPT_PHI0 = 1,        /* initial phi of Theorem 1's loop, as value/1024 (default 1280 = 1.25) */
    DM_OPT_COUNTERS = 2,    /* device pointer to uint64[4] accumulating areas inspected, darts
                               generated, darts kept and passes (0 = off) */
    DM_OPT_FORM = 3,        /* launch form: 0 = batched (default: sets classified by first rank
                               limit and binned by a Lemma 2 estimate of their work, costliest
                               first, persistent warps claiming work,
                               a block of 8 warps for each set of >= DM_OPT_LARGE_NNZ elements);
                               1 = plain (one warp per set in input order, static grid);
                               2 = persistent warps over the sets in input order */
    DM_OPT_WARPS_PER_BLOCK = 4, /* 1..8 warps (sets) per thread block, 0 = automatic */
    DM_OPT_LSH_PHI0 = 5,        /* initial phi of dm_lsh's loop, as value/1024 (default 3072 = 3.0) */
    DM_OPT_LARGE_NNZ = 6,       /* batched form: element count from which a set gets a whole block of
                                   8 warps (default 2048; 0 = never; dm_lsh never does).  A set of
                                   fewer than 512 elements on a block has each tile's areas split
                                   among the 8 warps; a larger one has its tiles dealt to them */
    DM_OPT_GRAPH = 7,           /* 1: launch each call's kernel sequence as a CUDA graph, cached per
                                   context; a call identical to a cached one (same pointers, sizes,
                                   seed and settings) replays it with one launch, a new call of the
                                   same shape patches the least recently used executable in place.
                                   Capture runs on a context-owned stream, so the caller's stream
                                   may itself be under capture.  0 (default): plain launches. */
    DM_OPT_TUNED = 8,           /* 1 (default): calls use the settings dm_autotune stored for their
                                   (kind, k, K, b), in place of the options above; 0: ignore them;
                                   2: forget them */
    DM_OPT_LARGE_WORK = 9,      /* batched form: a set whose Lemma 2 estimate of the areas it
                                   inspects (phi0 t + sum_i (log2(1 + t x_i) + 1) +
                                   nnz log2(1 + phi0/|x|_1)) reaches this value also gets a block of
                                   8 warps (default 0 = never; dm_lsh never does) */
    DM_OPT_HOST_CHUNKS = 10,    /* dm_sketch_host: number of chunks (1..256, default 8) a batch is
                                   split into, so that one chunk's copies overlap another's kernels
                                   (chunks hold at least 4,096 sets) */
    DM_OPT_HOST_MODE = 11,      /* dm_sketch_host: 0 = staged (chunked copies to device buffers);
                                   1 = in place (the kernels read the input arrays and write the
                                   outputs through the device's mapping of page-locked host memory,
                                   so the transfers ride on the kernels' own loads and stores; the
                                   call fails with DM_EINVAL if an array is not mapped); 2 (default)
                                   = in place when every array is page-locked and mapped, else staged */
    DM_OPT_SLOTS = 12           /* sketches: where the k bucket minima live while a set is sketched.
                                   0 (default) = automatic (the row layout when keys are written
                                   to device memory, else shared memory); 1 = shared
                                   memory (k 64-bit minima per warp); 2 = the output row (shared
                                   memory holds a 16-bit filter per bucket, the high half of a
                                   rank code already in the bucket's minimum; the 64-bit minimum
                                   is taken with an atomic minimum on the key in the output row;
                                   needs out_keys in device memory, else the call falls back to
                                   shared memory).  The choice never changes an output bit. */
};
int dm_set_option(dm_ctx *ctx, int option, int64_t value);

/* The settings dm_autotune chose and what they measured. */
typedef struct dm_tuning {
    int32_t form;             /* DM_OPT_FORM value (0 batched or 2 persistent) */
    int32_t warps_per_block;  /* warps per block actually used */
    int32_t phi0_1024;        /* initial phi, as value/1024 */
    int32_t large_nnz;        /* DM_OPT_LARGE_NNZ value */
    int32_t large_work;       /* DM_OPT_LARGE_WORK value */
    int64_t sets_timed;       /* rows of the batch the trials ran on */
    float ms_default;         /* median time of the trial batch with the context's options */
    float ms_tuned;           /* median time with the chosen settings */
    int32_t slots;            /* DM_OPT_SLOTS value */
} dm_tuning;

/* Launch-setting search (the paper has no counterpart; results never depend on the choice).
 * Runs the call that dm_sketch / dm_sketch_bbit (lsh = 0, K_or_b = b, 0 for keys only), dm_lsh
 * (lsh = 1, k = L, K_or_b = K) or dm_bottomk (lsh = 2, K_or_b = 0) would make on the first min(n_sets, max_sets) rows (max_sets <= 0:
 * 65536) of the given device batch, timing each candidate with CUDA events on `stream` (median of
 * three runs after a warm-up): initial phi, then warps per block, then the large-set threshold,
 * then the form, then (sketches with keys) the slot storage, each kept when it is faster.  Outputs of the trials go to temporary device
 * memory (counted against the budget); the caller's batch is only read.  The choice is stored in
 * the context for later calls with the same (kind, k, K, b) (see DM_OPT_TUNED) and, when result is
 * not NULL, written there.  Synchronous.  Returns DM_EINVAL for n_sets == 0 or bad arguments and
 * the first kernel-recorded error of the trial runs (a bad weight) like dm_sync_status. */
int dm_autotune(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                int64_t n_sets, int32_t lsh, int32_t k, int32_t K_or_b, uint64_t seed, int64_t max_sets,
                dm_tuning *result, void *stream);

/* Stores launch settings for later calls with the same (kind, k, K, b), exactly as dm_autotune
 * stores its choice (lsh, k and K_or_b as there), so that settings saved from an earlier
 * dm_autotune on this GPU model can be reinstalled without timing again.  Reads form,
 * warps_per_block (0 = automatic), phi0_1024, large_nnz and large_work; the other fields are
 * ignored.  Results never depend on the settings.  DM_EINVAL for values outside the options'
 * ranges. */
int dm_set_tuning(dm_ctx *ctx, int32_t lsh, int32_t k, int32_t K_or_b, const dm_tuning *tuning);

/* t = ceil(k ln k) + k as the library computes it (Theorem 1's proof); 0 for k < 1. */
int64_t dm_t_of_k(int32_t k);

/* The Poisson(1) inversion thresholds the library uses: T[n] = ceil(2^32 P(Poi(1) <= n)),
 * n = 0..11, written to host array out[12]. */
void dm_poisson_thresholds(uint32_t *out);

/* ---------------------------------------------------------------------------------------
 * Serving loop (the paper has no counterpart: it sketches one set per call on a CPU).
 * Requests of one weighted set each, with their own k and seed, are admitted against a memory
 * budget and batched continuously onto several lanes (a lane = a CUDA stream with its own
 * device and page-locked host buffer): whenever a lane is free it takes the oldest pending
 * requests, groups them by (k, seed), copies them to the device in one transfer, sketches each
 * group in one launch sequence and copies the keys back in one transfer.  Each request receives
 * exactly the keys dm_sketch gives for its row alone.  All pointers here are HOST pointers.
 * Thread safety: submit / poll / wait / stats may be called from any number of host threads.
 * --------------------------------------------------------------------------------------- */
typedef struct dm_server dm_server;

typedef struct dm_server_config {
    int32_t device;            /* CUDA device */
    int32_t lanes;             /* batches in flight at once (streams), 1..64; 0 = 4 */
    size_t mem_budget_bytes;   /* admission budget: device bytes of admitted, unfinished requests
                                  (32 + 8 nnz + 8 k each); 0 = 8 GiB.  The lanes' buffers are also
                                  kept within it */
    size_t lane_bytes;         /* device (and page-locked host) buffer of each lane = the largest
                                  batch; 0 = min(budget / lanes, 64 MiB) */
    int32_t max_batch;         /* requests per batch; 0 = 4096 */
    int32_t max_wait_us;       /* batching window: a free lane waits until the oldest pending
                                  request is this old (or the batch is full); 0 = no wait */
    int32_t per_request;       /* 1 = plain per-request form (one request per batch, plain launch):
                                  the comparison the batching is measured against */
    int32_t large_nnz;         /* a group with a set of at least this many elements runs the batched
                                  form (a block per such set); other groups run persistent warps;
                                  0 = 2048 */
} dm_server_config;

typedef struct dm_server_stats {
    int64_t submitted;         /* admitted requests */
    int64_t completed;         /* finished requests (including failed ones) */
    int64_t failed;            /* finished with a non-zero status */
    int64_t rejected;          /* DM_EAGAIN answers */
    int64_t batches;
    int64_t admitted_bytes;    /* currently admitted */
    double mean_batch;         /* requests per batch */
    double p50_us, p99_us, max_us;   /* latency from arrival to result ready, over the most recent
                                        4,194,304 completions */
    int64_t groups;            /* (k, seed) groups run: one launch sequence each */
    int64_t kernel_launches;   /* kernels launched for them (since the server started) */
} dm_server_stats;

/* Start a server: creates the lanes (contexts, streams, buffers) and one worker thread per lane.
 * DM_EINVAL for a bad configuration, DM_ENOMEM if the buffers cannot be allocated. */
int dm_server_create(dm_server **out, const dm_server_config *cfg);

/* Finish every admitted request, stop the workers and release everything. */
int dm_server_destroy(dm_server *srv);

/* Submit one set (indices uint32[nnz], weights float32[nnz], host memory; both are copied before
 * the call returns) for k minhashes with `seed`.  The keys are written to out (host uint64[k],
 * which must stay valid until the request is reported done; NULL = computed but not delivered).
 * On DM_OK *ticket identifies the request for dm_server_poll / dm_server_wait, one of which must
 * eventually report it done (that releases it).  DM_EAGAIN: the budget is full now (nothing was
 * admitted; retry).  DM_EINVAL: bad k or a negative, NaN or infinite weight.  DM_ENOMEM: the
 * request alone is larger than a lane. */
int dm_server_submit(dm_server *srv, const uint32_t *indices, const float *weights, int64_t nnz, int32_t k,
                     uint64_t seed, uint64_t *out, int64_t *ticket);

/* Without blocking: *status = -1 while the request is pending, else its final status (DM_OK, or
 * the error its batch or its row met), in which case the ticket is released.  Returns DM_EINVAL for
 * an unknown or released ticket. */
int dm_server_poll(dm_server *srv, int64_t ticket, int32_t *status);

/* Block until the request is done (timeout_us < 0: no limit) and release the ticket; *status as
 * for dm_server_poll.  Returns DM_ETIMEOUT if the limit passed first (the ticket stays valid). */
int dm_server_wait(dm_server *srv, int64_t ticket, int64_t timeout_us, int32_t *status);

/* Play a request trace in real time from the calling thread: request i (row i of the CSR
 * indptr/indices/weights, k[i], seed[i]) is submitted arrival_ns[i] nanoseconds after the start
 * (non-decreasing); one refused for lack of budget is resubmitted as capacity frees.  Returns when
 * all are done.  out (NULL = not delivered) receives the keys of request i at offset
 * k[0] + ... + k[i-1]; latency_ns[i] (may be NULL) the time from the scheduled arrival to result
 * ready; status[i] (may be NULL) the request's status (requests failing the host checks get
 * DM_EINVAL and latency 0 without being submitted). */
int dm_server_replay(dm_server *srv, int64_t n, const int64_t *indptr, const uint32_t *indices,
                     const float *weights, const int32_t *k, const uint64_t *seed, const int64_t *arrival_ns,
                     uint64_t *out, int64_t *latency_ns, int32_t *status);

int dm_server_get_stats(dm_server *srv, dm_server_stats *out);
int dm_server_reset_stats(dm_server *srv);

/* Host-side fault injection: the next `batches` batches fail before any GPU work is queued, as a
 * failed launch would; their requests finish with DM_ECUDA and the server carries on. */
int dm_server_fail_batches(dm_server *srv, int32_t batches);

#ifdef __cplusplus
}
#endif
#endif /* DARTMINHASH_H */
