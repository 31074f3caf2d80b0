// C ABI of libdartminhash.so (declared in include/dartminhash.h).
//
// Host responsibilities: argument checks, the per-k constant t = ceil(k ln k) + k of
// Theorem 1's proof, the Poisson(1) inversion table used by Algorithm 1 (computed here in
// exact fixed point, uploaded to __constant__ memory), launch configuration, the
// device-side status word and the host-buffer staging path.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "dm_device.cuh"
#include "dm_internal.h"

using dm::SketchParams;

struct dm_ctx {
    int device = 0;
    size_t budget = 0;
    int sm_count = 0;
    int *d_status = nullptr;
    int *h_status = nullptr;       // pinned
    float phi0 = 1.0f;             // initial phi of the sketch loop (Theorem 1)
    float phi0_lsh = 4.0f;         // initial phi of the LSH loop (every bucket needs K darts)
    unsigned long long *counters = nullptr;
    int form = 0;                  // 0 batched, 1 plain, 2 persistent in input order
    int warps_per_block = 0;       // 0 = automatic
    int large_nnz = 2048;          // batched form: sets with this many elements get a block
    // staging for the host-buffer entry points
    void *d_stage = nullptr;
    size_t d_stage_bytes = 0;
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr;
    // general-kernel work queue for calls on device buffers: int32[queue_cap] + a counter
    void *d_queue = nullptr;
    int64_t queue_cap = 0;
};

namespace {

// t = ceil(k ln k) + k.  The product k ln k is irrational for k >= 2; double precision decides
// the ceiling whenever k ln k is farther than 1e-6 from an integer, which holds for every
// k <= 8192 (the supported range); otherwise 0 is returned and the call is rejected.
int64_t t_of_k(int32_t k) {
    if (k < 1) return 0;
    if (k == 1) return 1;
    double v = (double)k * std::log((double)k);
    double c = std::ceil(v);
    if (c - v < 1e-6 || v - (c - 1.0) < 1e-6) return 0;
    return (int64_t)c + k;
}

// T[n] = ceil(2^32 P(Poi(1) <= n)) = ceil(2^32 e^-1 sum_{m<=n} 1/m!), n = 0..11.
// e^-1 and the partial sums are formed in 2^-96 fixed point with unsigned 128-bit integers;
// every rounding is bounded, and the ceiling is only accepted when the value is at least 2^-20
// away from an integer (it is, by far, for every n).
bool poisson_table(uint32_t *T) {
    typedef unsigned __int128 u128;
    const int FB = 96;
    const u128 ONE = (u128)1 << FB;
    // inverse factorials 1/m! (floor), m = 0..40
    u128 invf[41];
    invf[0] = ONE;
    for (int m = 1; m <= 40; ++m) invf[m] = invf[m - 1] / (u128)m;
    // e^-1 = sum (-1)^m / m!  (each term floored: total error < 41 * 2^-96)
    u128 pos = 0, neg = 0;
    for (int m = 0; m <= 40; ++m) (m % 2 ? neg : pos) += invf[m];
    u128 einv = pos - neg;
    u128 cum = 0;
    for (int n = 0; n < 12; ++n) {
        cum += invf[n];
        // 2^32 e^-1 cum: e^-1 in 2^-64 fixed point (< 2^64), cum in 2^-62 fixed point (< 2^64,
        // cum < e), product in 2^-126 fixed point, so the value is prod / 2^94.  Truncation
        // error is below 2^-28 in units of the result; demand 2^-20 clearance from an integer.
        u128 a = einv >> 32, b = cum >> 34;
        u128 prod = a * b;
        u128 ip = prod >> 94;
        u128 frac = prod & (((u128)1 << 94) - 1);
        u128 margin = (u128)1 << 74;
        if (frac < margin || frac > (((u128)1 << 94) - margin)) return false;
        uint64_t v = (uint64_t)ip + 1;
        if (v >= (1ull << 32)) return false;
        T[n] = (uint32_t)v;
    }
    return true;
}

bool g_table_ok = false;
uint32_t g_table[12];
std::once_flag g_table_once;

const uint32_t *table() {
    std::call_once(g_table_once, [] { g_table_ok = poisson_table(g_table); });
    return g_table_ok ? g_table : nullptr;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return DM_OK;
    return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
}

// Warps per block: as many as fit 96 KB of shared memory (so two or more blocks are resident),
// at most 8.
int auto_warps(bool lsh, int k, int K) {
    size_t a = dm::warp_bytes(lsh, k, K, 0), b = dm::warp_bytes(lsh, k, K, 1);
    size_t per = a > b ? a : b;
    int w = (int)((96 * 1024) / per);
    if (w > 8) w = 8;
    if (w < 1) w = 1;
    return w;
}

int check_csr(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n) {
    if (n < 0) return DM_EINVAL;
    if (n > 0 && (!indptr || !indices || !weights)) return DM_EINVAL;
    return DM_OK;
}

// Scratch of a call of n_sets sets: work queue, order, classes and counters.
size_t queue_bytes(int64_t n_sets) { return dm::call_scratch_bytes(n_sets); }

int ensure_queue(dm_ctx *ctx, int64_t n_sets) {
    if (n_sets <= ctx->queue_cap) return DM_OK;
    size_t need = queue_bytes(n_sets);
    if (ctx->budget && need + ctx->d_stage_bytes > ctx->budget) return DM_ENOMEM;
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    ctx->d_queue = nullptr;
    ctx->queue_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->d_queue, need);
    if (e != cudaSuccess) return cuda_fail(e);
    ctx->queue_cap = n_sets;
    return DM_OK;
}

// One batched call: sketches (lsh = false: k minhashes, optional b-bit words) or (L, K) LSH
// (lsh = true: k = L).  queue: scratch for the general kernel's work queue (null = context's).
int run_sets(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
             int64_t n_sets, bool lsh, int32_t k, int32_t K, int32_t b, uint64_t seed, uint64_t *out_words,
             uint64_t *out_keys, uint32_t *out_lsh, cudaStream_t st, void *queue = nullptr) {
    if (!ctx) return DM_EINVAL;
    int rc = check_csr(indptr, indices, weights, n_sets);
    if (rc) return rc;
    int64_t t;
    if (lsh) {
        if (k < 1 || k > 1024 || K < 1 || K > 32 || !out_lsh) return DM_EINVAL;
        t = (int64_t)k * K;
    } else {
        if (k < 1 || k > 8192) return DM_EINVAL;
        t = t_of_k(k);
        if (t <= 0) return DM_EINVAL;
    }
    bool bbit = b > 0;
    if (bbit && !(b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32)) return DM_EINVAL;
    if (!lsh && !bbit && !out_keys) return DM_EINVAL;
    if (bbit && !out_words) return DM_EINVAL;
    if (n_sets == 0) return DM_OK;
    if (n_sets > 0x7FFFFFFF) return DM_EINVAL;
    const int wpb = ctx->warps_per_block > 0 ? ctx->warps_per_block : auto_warps(lsh, k, K);
    const size_t smem_fast = dm::warp_bytes(lsh, k, K, 0) * wpb, smem = dm::warp_bytes(lsh, k, K, 1) * wpb;
    if (smem > 227 * 1024 || smem_fast > 227 * 1024) return DM_EINVAL;     // L and K too large for LSH
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!queue) {
        if ((rc = ensure_queue(ctx, n_sets)) != DM_OK) return rc;
        queue = ctx->d_queue;
    }
    SketchParams p;
    std::memset(&p, 0, sizeof(p));
    p.indptr = indptr;
    p.indices = indices;
    p.weights = weights;
    p.n_sets = n_sets;
    p.k = k;
    p.K = lsh ? K : 0;
    p.t = (uint32_t)t;
    p.sigma = dm::mix64(seed ^ dm::kSeedSalt);
    p.phi0 = lsh ? ctx->phi0_lsh : ctx->phi0;
    p.b = bbit ? b : 0;
    p.words = bbit ? (int32_t)(((int64_t)k * b + 63) / 64) : 0;
    p.out_keys = out_keys;
    p.out_words = out_words;
    p.out_lsh = out_lsh;
    p.status = ctx->d_status;
    p.counters = ctx->counters;
    p.warps_per_block = wpb;
    p.warp_bytes = (int32_t)dm::warp_bytes(lsh, k, K, 1);
    p.warp_bytes_fast = (int32_t)dm::warp_bytes(lsh, k, K, 0);
    p.sink_bytes = (int32_t)dm::sink_bytes(lsh, k, K);
    dm::carve_call_scratch(queue, n_sets, p);
    const bool count = ctx->counters != nullptr;
    const int64_t blocks = (n_sets + wpb - 1) / wpb;
    if (ctx->form == 1) {
        // plain form: one warp per set in input order, a block per wpb sets
        p.sched = 1;
        return cuda_fail(dm::launch_sets(p, lsh, bbit, count, (int)blocks, (int)blocks, st));
    }
    // persistent grids: as many blocks as can be resident, never more than there are sets
    const int64_t cap0 = (int64_t)ctx->sm_count * dm::blocks_per_sm(lsh, 0, bbit, wpb, smem_fast);
    const int64_t cap1 = (int64_t)ctx->sm_count * dm::blocks_per_sm(lsh, 1, bbit, wpb, smem);
    const int grid = (int)(blocks < cap0 ? blocks : cap0);
    const int grid_general = (int)(blocks < cap1 ? blocks : cap1);
    if (ctx->form == 2) return cuda_fail(dm::launch_sets(p, lsh, bbit, count, grid, grid_general, st));
    // batched form (default): large sets get a block of 8 warps
    p.large_warps = 8;
    p.large_nnz = lsh ? 0 : ctx->large_nnz;
    int grid_large = 0;
    if (p.large_nnz > 0) {
        const size_t lb = dm::large_block_bytes(k, p.large_warps);
        if (lb <= 227 * 1024) grid_large = ctx->sm_count * dm::large_blocks_per_sm(bbit, p.large_warps, lb);
        else p.large_nnz = 0;
    }
    return cuda_fail(dm::launch_batched(p, lsh, bbit, count, grid, grid_general, grid_large, st));
}

int run_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
               int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words,
               uint64_t *out_keys, cudaStream_t st, void *queue = nullptr) {
    return run_sets(ctx, indptr, indices, weights, n_sets, false, k, 0, b, seed, out_words, out_keys, nullptr,
                    st, queue);
}

}  // namespace

extern "C" {

int dm_create(dm_ctx **out, int device, size_t mem_budget_bytes) {
    if (!out) return DM_EINVAL;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e);
    if (device < 0 || device >= n) return DM_EINVAL;
    const uint32_t *T = table();
    if (!T) return DM_EINVAL;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e);
    dm_ctx *c = new dm_ctx();
    c->device = device;
    c->budget = mem_budget_bytes;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if ((e = cudaMalloc(&c->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(c->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_status, sizeof(int))) != cudaSuccess ||
        (e = dm::upload_poisson_table(T)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        dm_destroy(c);
        return cuda_fail(e);
    }
    *out = c;
    return DM_OK;
}

int dm_destroy(dm_ctx *ctx) {
    if (!ctx) return DM_OK;
    cudaSetDevice(ctx->device);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    for (int i = 0; i < 2; ++i)
        if (ctx->copy_stream[i]) cudaStreamDestroy(ctx->copy_stream[i]);
    if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
    delete ctx;
    return DM_OK;
}

int dm_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
              int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream) {
    return run_sketch(ctx, indptr, indices, weights, n_sets, k, 0, seed, nullptr, out, (cudaStream_t)stream);
}

int dm_sketch_bbit(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                   int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words,
                   uint64_t *out_keys, void *stream) {
    if (b <= 0) return DM_EINVAL;
    return run_sketch(ctx, indptr, indices, weights, n_sets, k, b, seed, out_words, out_keys,
                      (cudaStream_t)stream);
}

int dm_lsh(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
           int64_t n_sets, int32_t L, int32_t K, uint64_t seed, uint32_t *out, void *stream) {
    return run_sets(ctx, indptr, indices, weights, n_sets, true, L, K, 0, seed, nullptr, nullptr, out,
                    (cudaStream_t)stream);
}

int dm_sketch_host(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                   int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_keys,
                   uint64_t *out_words, void *stream) {
    if (!ctx) return DM_EINVAL;
    int rc = check_csr(indptr, indices, weights, n_sets);
    if (rc) return rc;
    if (k < 1 || k > 8192) return DM_EINVAL;
    if (b < 0 || (b == 0 && !out_keys) || (b > 0 && !out_words)) return DM_EINVAL;
    if (n_sets == 0) return DM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e);
    if (indptr[0] != 0 || indptr[n_sets] < 0) return DM_EINVAL;
    const int64_t words = b > 0 ? ((int64_t)k * b + 63) / 64 : 0;
    // chunks of about 1/8 of the batch (at least 16k sets), two buffer sets in flight
    int64_t cs = (n_sets + 7) / 8;
    if (cs < 16384) cs = 16384;
    if (cs > n_sets) cs = n_sets;
    int64_t max_nnz = 0;
    for (int64_t s0 = 0; s0 < n_sets; s0 += cs) {
        int64_t s1 = s0 + cs < n_sets ? s0 + cs : n_sets;
        int64_t z = indptr[s1] - indptr[s0];
        if (z < 0) return DM_EINVAL;
        if (z > max_nnz) max_nnz = z;
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_ip = al((size_t)(cs + 1) * 8), b_ix = al((size_t)max_nnz * 4), b_w = b_ix;
    const size_t b_keys = out_keys ? al((size_t)cs * k * 8) : 0, b_words = al((size_t)cs * words * 8);
    const size_t b_q = queue_bytes(cs);
    const size_t per = b_ip + b_ix + b_w + b_keys + b_words + b_q;
    const size_t need = 2 * per;
    if (need > ctx->d_stage_bytes) {
        if (ctx->budget && need > ctx->budget) return DM_ENOMEM;
        if (ctx->d_stage) cudaFree(ctx->d_stage);
        ctx->d_stage = nullptr;
        ctx->d_stage_bytes = 0;
        if ((e = cudaMalloc(&ctx->d_stage, need)) != cudaSuccess) return cuda_fail(e);
        ctx->d_stage_bytes = need;
    }
    if (!ctx->copy_stream[0]) {
        for (int i = 0; i < 2; ++i)
            if ((e = cudaStreamCreateWithFlags(&ctx->copy_stream[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e);
        if ((e = cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e);
    }
    // the staged work starts after everything already queued on the caller's stream
    if ((e = cudaEventRecord(ctx->ev_start, st)) != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamWaitEvent(ctx->copy_stream[i], ctx->ev_start, 0)) != cudaSuccess) return cuda_fail(e);
    int chunk = 0;
    for (int64_t s0 = 0; s0 < n_sets; s0 += cs, ++chunk) {
        const int64_t s1 = s0 + cs < n_sets ? s0 + cs : n_sets, n = s1 - s0;
        const int64_t z0 = indptr[s0], z = indptr[s1] - z0;
        cudaStream_t cst = ctx->copy_stream[chunk & 1];
        char *base = (char *)ctx->d_stage + (size_t)(chunk & 1) * per;
        int64_t *d_ip = (int64_t *)base;
        uint32_t *d_ix = (uint32_t *)(base + b_ip);
        float *d_w = (float *)(base + b_ip + b_ix);
        uint64_t *d_keys = out_keys ? (uint64_t *)(base + b_ip + b_ix + b_w) : nullptr;
        uint64_t *d_words = (uint64_t *)(base + b_ip + b_ix + b_w + b_keys);
        void *d_q = base + b_ip + b_ix + b_w + b_keys + b_words;
        // indptr keeps absolute offsets; the element arrays are addressed from z0
        if ((e = cudaMemcpyAsync(d_ip, indptr + s0, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, cst)) ||
            (z && (e = cudaMemcpyAsync(d_ix, indices + z0, (size_t)z * 4, cudaMemcpyHostToDevice, cst))) ||
            (z && (e = cudaMemcpyAsync(d_w, weights + z0, (size_t)z * 4, cudaMemcpyHostToDevice, cst))))
            return cuda_fail(e);
        rc = run_sketch(ctx, d_ip, d_ix - z0, d_w - z0, n, k, b, seed, b > 0 ? d_words : nullptr,
                        d_keys, cst, d_q);
        if (rc) return rc;
        if ((out_keys && (e = cudaMemcpyAsync(out_keys + s0 * k, d_keys, (size_t)n * k * 8,
                                              cudaMemcpyDeviceToHost, cst))) ||
            (b > 0 && (e = cudaMemcpyAsync(out_words + s0 * words, d_words, (size_t)n * words * 8,
                                           cudaMemcpyDeviceToHost, cst))))
            return cuda_fail(e);
    }
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamSynchronize(ctx->copy_stream[i])) != cudaSuccess) return cuda_fail(e);
    return DM_OK;
}

int dm_sync_status(dm_ctx *ctx, void *stream) {
    if (!ctx) return DM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DM_ECUDA;
    int s = *ctx->h_status;
    if (s) {
        e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DM_ECUDA;
    }
    return s;
}

const char *dm_strerror(int status) {
    switch (status) {
        case DM_OK: return "ok";
        case DM_EINVAL: return "invalid argument or weight";
        case DM_ENOMEM: return "out of memory or over the context's memory budget";
        case DM_ECUDA: return "CUDA runtime error";
        case DM_ETIMEOUT: return "bounded device wait gave up";
        case DM_ERANGE: return "input outside the supported numeric range";
        case DM_EOVERFLOW: return "rank-limit doubling reached its limit";
        default: return "unknown status";
    }
}

int dm_set_option(dm_ctx *ctx, int option, int64_t value) {
    if (!ctx) return DM_EINVAL;
    switch (option) {
        case DM_OPT_PHI0:
            if (value < 1 || value > 1024 * 1024) return DM_EINVAL;
            ctx->phi0 = (float)value / 1024.0f;
            return DM_OK;
        case DM_OPT_COUNTERS:
            ctx->counters = (unsigned long long *)(uintptr_t)value;
            return DM_OK;
        case DM_OPT_FORM:
            if (value < 0 || value > 2) return DM_EINVAL;
            ctx->form = (int)value;
            return DM_OK;
        case DM_OPT_LARGE_NNZ:
            if (value < 0 || value > 0x7FFFFFFF) return DM_EINVAL;
            ctx->large_nnz = (int)value;
            return DM_OK;
        case DM_OPT_LSH_PHI0:
            if (value < 1 || value > 1024 * 1024) return DM_EINVAL;
            ctx->phi0_lsh = (float)value / 1024.0f;
            return DM_OK;
        case DM_OPT_WARPS_PER_BLOCK:
            if (value < 0 || value > 8) return DM_EINVAL;   // kernels are built for <= 256 threads
            ctx->warps_per_block = (int)value;
            return DM_OK;
        default:
            return DM_EINVAL;
    }
}

int64_t dm_t_of_k(int32_t k) { return t_of_k(k); }

void dm_poisson_thresholds(uint32_t *out) {
    const uint32_t *T = table();
    for (int n = 0; n < 12; ++n) out[n] = T ? T[n] : 0;
}

}  // extern "C"
