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
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dm_device.cuh"
#include "dm_internal.h"

using dm::SketchParams;

namespace {

// Launch settings of one call.  None of them changes an output bit (the results are independent
// of phi0, the form and the launch shape); they only move work around.
struct Choice {
    int form;           // 0 batched, 1 plain, 2 persistent in input order
    int wpb;            // warps (sets) per block, 0 = automatic
    float phi0;         // initial phi of Theorem 1's loop
    int large_nnz;      // batched form: element count from which a set gets a whole block
    float large_work;   // batched form: Lemma 2 work estimate from which a set gets one (0: off)
    int slots;          // sketch bucket minima: 0 automatic, 1 shared memory, 2 the output row
};

struct TunedEntry {
    int kind;
    int k, K, b;
    Choice c;
};

// Everything a call's launch sequence depends on.  Built zero-filled (padding included) so two
// plans compare equal with memcmp exactly when the launches would be identical.
struct Plan {
    SketchParams p;
    int kind, bbit, count, form, grid_fast, grid_general, grid_large;
};

struct GraphEntry {
    Plan plan;
    cudaGraphExec_t exec;
    uint64_t used;
};

constexpr size_t kMaxGraphs = 16;

}  // namespace

struct dm_ctx {
    int device = 0;
    size_t budget = 0;
    int sm_count = 0;
    int *d_status = nullptr;
    int *h_status = nullptr;       // pinned
    float phi0 = dm::kDefaultPhi0; // initial phi of the sketch loop (Theorem 1)
    float phi0_lsh = 3.0f;         // initial phi of the LSH loop (every bucket needs K darts)
    unsigned long long *counters = nullptr;
    int form = 0;                  // 0 batched, 1 plain, 2 persistent in input order
    int warps_per_block = 0;       // 0 = automatic
    int large_nnz = 2048;          // batched form: sets with this many elements get a block
    float large_work = 0.f;        // batched form: sets with this work estimate get a block
    int slots = 0;                 // sketch bucket minima: 0 automatic, 1 shared memory, 2 output row
    int host_chunks = 8;           // host-buffer entry: chunks a batch is split into
    int host_mode = 2;             // host-buffer entry: 0 staged, 1 in place, 2 in place when possible
    bool host_out = false;         // the current call writes host memory in place: no key-row layout
    // staging for the host-buffer entry points
    void *d_stage = nullptr;
    size_t d_stage_bytes = 0;
    cudaStream_t copy_stream[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr;
    // general-kernel work queue for calls on device buffers: int32[queue_cap] + a counter
    void *d_queue = nullptr;
    int64_t queue_cap = 0;
    // launch settings that dm_autotune chose, per (kind, k, K, b)
    std::vector<TunedEntry> tuned;
    bool use_tuned = true;
    // CUDA-graph replay of repeated identical calls
    bool use_graph = false;
    std::vector<GraphEntry> graphs;
    uint64_t graph_tick = 0;
    cudaStream_t capture_stream = nullptr;
    // resident blocks per SM, per kernel and launch shape
    std::vector<std::pair<uint64_t, int>> occupancy;
    // side stream of the batched form's large-set and general kernels (created on first use)
    dm::SideStream side = {nullptr, nullptr, nullptr};
    bool side_ready = false;
};

namespace {

// NVTX range around a library call, for timelines (a no-op unless a tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

const char *kind_name(int kind) {
    return kind == dm::kLsh ? "dm_lsh" : (kind == dm::kBottomK ? "dm_bottomk" : "dm_sketch");
}

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
int auto_warps(int kind, int k, int K, bool key_row = false) {
    size_t a = dm::warp_bytes(kind, k, K, 0, key_row), b = dm::warp_bytes(kind, k, K, 1, key_row);
    size_t per = a > b ? a : b;
    int w = (int)((96 * 1024) / per);
    if (w > 8) w = 8;
    if (w < 1) w = 1;
    return w;
}

int check_csr(const int64_t *indptr, const uint32_t *indices, const float *weights, int64_t n) {
    if (n < 0) return DM_EINVAL;
    if (n > 0 && (!indptr || !indices || !weights)) return DM_EINVAL;
    // every array aligned to its element size (a misaligned load would fault on the device)
    if (((uintptr_t)indptr & 7u) || ((uintptr_t)indices & 3u) || ((uintptr_t)weights & 3u)) return DM_EINVAL;
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

// Blocks of a kernel resident per SM, cached per context (the query costs a few microseconds).
// which: 0 fast, 1 general, 2 large.
int occupancy(dm_ctx *ctx, int which, int kind, bool bbit, int wpb, size_t smem, bool key_row) {
    const uint64_t key = ((uint64_t)which) | ((uint64_t)kind << 2) | ((uint64_t)bbit << 4) |
                         ((uint64_t)key_row << 5) | ((uint64_t)wpb << 6) | ((uint64_t)smem << 12);
    for (auto &e : ctx->occupancy)
        if (e.first == key) return e.second;
    int nb = which == 2 ? dm::large_blocks_per_sm(bbit, wpb, smem, key_row)
                        : dm::blocks_per_sm(kind, which, bbit, wpb, smem, key_row);
    ctx->occupancy.emplace_back(key, nb);
    return nb;
}

Choice choose(const dm_ctx *ctx, int kind, int k, int K, int b) {
    Choice c{ctx->form, ctx->warps_per_block, kind == dm::kLsh ? ctx->phi0_lsh : ctx->phi0, ctx->large_nnz,
             ctx->large_work, ctx->slots};
    if (ctx->use_tuned)
        for (const auto &e : ctx->tuned)
            if (e.kind == kind && e.k == k && e.K == K && e.b == b) return e.c;
    return c;
}

// Checks a call and fills its plan: sketches (kSketch: k minhashes, optional b-bit words), (L, K)
// LSH (kLsh: k = L) or bottom-k sketches (kBottomK: the k smallest keys).  queue: scratch for the
// call's work queue (null = the context's).  Returns DM_OK with pl.p.n_sets == 0 when there is
// nothing to launch.
int plan_call(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
              int64_t n_sets, int kind, int32_t k, int32_t K, int32_t b, uint64_t seed, uint64_t *out_words,
              uint64_t *out_keys, uint32_t *out_lsh, void *queue, const Choice &ch, Plan &pl,
              const int32_t *scale = nullptr) {
    const bool lsh = kind == dm::kLsh;
    std::memset(&pl, 0, sizeof(pl));
    if (!ctx) return DM_EINVAL;
    int rc = check_csr(indptr, indices, weights, n_sets);
    if (rc) return rc;
    int64_t t;
    if (lsh) {
        if (k < 1 || k > 1024 || K < 1 || K > 32 || !out_lsh) return DM_EINVAL;
        t = (int64_t)k * K;
    } else if (kind == dm::kBottomK) {
        if (k < 1 || k > 1024 || !out_keys || b != 0) return DM_EINVAL;
        t = k;                                      // Section 3: t = k for the bottom-k sketch
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
    // sketches with keys in device memory keep their minima in the output row (a 16-bit filter
    // per bucket in shared memory) unless DM_OPT_SLOTS asks for shared minima
    const bool row_ok = kind == dm::kSketch && out_keys && !ctx->host_out;
    const bool key_row = row_ok && ch.slots != 1;
    const int wpb = ch.wpb > 0 ? ch.wpb : auto_warps(kind, k, K, key_row);
    const size_t smem_fast = dm::warp_bytes(kind, k, K, 0, key_row) * wpb,
                 smem = dm::warp_bytes(kind, k, K, 1, key_row) * wpb;
    if (smem > 227 * 1024 || smem_fast > 227 * 1024) return DM_EINVAL;     // L and K too large for LSH
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!queue) {
        if ((rc = ensure_queue(ctx, n_sets)) != DM_OK) return rc;
        queue = ctx->d_queue;
    }
    SketchParams &p = pl.p;
    p.indptr = indptr;
    p.indices = indices;
    p.weights = weights;
    p.n_sets = n_sets;
    p.k = k;
    p.K = lsh ? K : 0;
    p.t = (uint32_t)t;
    p.sigma = dm::mix64(seed ^ dm::kSeedSalt);
    p.phi0 = ch.phi0;
    p.scale = scale;
    p.b = bbit ? b : 0;
    p.words = bbit ? (int32_t)(((int64_t)k * b + 63) / 64) : 0;
    p.out_keys = out_keys;
    p.out_words = out_words;
    p.out_lsh = out_lsh;
    p.status = ctx->d_status;
    p.counters = ctx->counters;
    p.warps_per_block = wpb;
    p.warp_bytes = (int32_t)dm::warp_bytes(kind, k, K, 1, key_row);
    p.warp_bytes_fast = (int32_t)dm::warp_bytes(kind, k, K, 0, key_row);
    p.sink_bytes = (int32_t)((dm::sink_bytes(kind, k, K, key_row) + 15) & ~(size_t)15);
    p.key_row = key_row;
    dm::carve_call_scratch(queue, n_sets, p);
    pl.kind = kind;
    pl.bbit = bbit;
    pl.count = ctx->counters != nullptr;
    pl.form = ch.form;
    const int64_t blocks = (n_sets + wpb - 1) / wpb;
    if (ch.form == 1) {
        // plain form: one warp per set in input order, a block per wpb sets
        p.sched = 1;
        pl.grid_fast = pl.grid_general = (int)blocks;
        return DM_OK;
    }
    // persistent grids: as many blocks as can be resident, never more than there are sets
    const int64_t cap0 = (int64_t)ctx->sm_count * occupancy(ctx, 0, kind, bbit, wpb, smem_fast, key_row);
    const int64_t cap1 = (int64_t)ctx->sm_count * occupancy(ctx, 1, kind, bbit, wpb, smem, key_row);
    pl.grid_fast = (int)(blocks < cap0 ? blocks : cap0);
    pl.grid_general = (int)(blocks < cap1 ? blocks : cap1);
    if (ch.form == 2) return DM_OK;
    // batched form (default): large sets get a block of 8 warps
    p.large_warps = 8;
    p.large_nnz = kind != dm::kSketch ? 0 : ch.large_nnz;
    p.large_work = kind != dm::kSketch ? 0.f : ch.large_work;
    if (p.large_nnz > 0 || p.large_work > 0.f) {
        const size_t lb = dm::large_block_bytes(k, p.large_warps, key_row);
        if (lb <= 227 * 1024) pl.grid_large = ctx->sm_count * occupancy(ctx, 2, dm::kSketch, bbit, p.large_warps, lb, key_row);
        else p.large_nnz = 0;
    }
    return DM_OK;
}

cudaError_t ensure_side(dm_ctx *ctx) {
    if (ctx->side_ready) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&ctx->side.st, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->side.join, cudaEventDisableTiming)) != cudaSuccess)
        return e;
    ctx->side_ready = true;
    return cudaSuccess;
}

cudaError_t launch_plan(dm_ctx *ctx, const Plan &pl, cudaStream_t st) {
    if (pl.form == 0) {
        // the side stream carries the large-set kernel and the general kernel beside the fast one
        cudaError_t e = ensure_side(ctx);
        if (e != cudaSuccess) return e;
        const dm::SideStream *side = &ctx->side;
        return dm::launch_batched(pl.p, pl.kind, pl.bbit, pl.count, pl.grid_fast, pl.grid_general, pl.grid_large, st,
                                  side);
    }
    return dm::launch_sets(pl.p, pl.kind, pl.bbit, pl.count, pl.grid_fast, pl.grid_general, st);
}

void drop_graphs(dm_ctx *ctx) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

// Launches a plan, directly or (graph replay on) from a cached graph executable.  A plan seen
// before is replayed as is; a new plan is captured on the context's capture stream and either
// patched into the least recently used executable (when its launch sequence has the same
// shape) or instantiated, the cache holding at most kMaxGraphs.
int run_plan(dm_ctx *ctx, const Plan &pl, cudaStream_t st) {
    if (!ctx->use_graph) return cuda_fail(launch_plan(ctx, pl, st));
    for (auto &g : ctx->graphs)
        if (std::memcmp(&g.plan, &pl, sizeof(Plan)) == 0) {
            g.used = ++ctx->graph_tick;
            return cuda_fail(cudaGraphLaunch(g.exec, st));
        }
    cudaError_t e;
    if (!ctx->capture_stream &&
        (e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaError_t el = launch_plan(ctx, pl, ctx->capture_stream);
    e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (el != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(el != cudaSuccess ? el : e);
    }
    // same shape: same kernels in the same order (form, kind, templates, large kernel on/off)
    auto same_shape = [&](const Plan &a) {
        return a.form == pl.form && a.kind == pl.kind && a.bbit == pl.bbit && a.count == pl.count &&
               (a.grid_large > 0 && (a.p.large_nnz > 0 || a.p.large_work > 0.f)) ==
                   (pl.grid_large > 0 && (pl.p.large_nnz > 0 || pl.p.large_work > 0.f));
    };
    GraphEntry *slot = nullptr;
    for (auto &g : ctx->graphs)
        if (same_shape(g.plan) && (!slot || g.used < slot->used)) slot = &g;
    bool ready = false;
    if (slot) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(slot->exec, graph, &info) == cudaSuccess) ready = true;
        else cudaGetLastError();      // clear the update's error; instantiate below instead
    }
    if (!ready) {
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(e);
        }
        if (ctx->graphs.size() >= kMaxGraphs) {
            slot = &ctx->graphs[0];
            for (auto &g : ctx->graphs)
                if (g.used < slot->used) slot = &g;
            cudaGraphExecDestroy(slot->exec);
        } else {
            ctx->graphs.push_back(GraphEntry{});
            slot = &ctx->graphs.back();
        }
        slot->exec = exec;
    }
    cudaGraphDestroy(graph);
    std::memcpy(&slot->plan, &pl, sizeof(Plan));
    slot->used = ++ctx->graph_tick;
    return cuda_fail(cudaGraphLaunch(slot->exec, st));
}

int run_sets(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
             int64_t n_sets, int kind, int32_t k, int32_t K, int32_t b, uint64_t seed, uint64_t *out_words,
             uint64_t *out_keys, uint32_t *out_lsh, cudaStream_t st, void *queue = nullptr,
             const Choice *force = nullptr, const int32_t *scale = nullptr) {
    if (!ctx) return DM_EINVAL;
    Range range(kind_name(kind));
    const Choice ch = force ? *force : choose(ctx, kind, k, K, b);
    Plan pl;
    int rc = plan_call(ctx, indptr, indices, weights, n_sets, kind, k, K, b, seed, out_words, out_keys, out_lsh,
                       queue, ch, pl, scale);
    if (rc || pl.p.n_sets == 0) return rc;
    return run_plan(ctx, pl, st);
}

}  // namespace

// Helpers of the serving loop (declared in dm_internal.h).
namespace dm {

int serve_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                 int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *queue, int form, int large_nnz,
                 cudaStream_t st) {
    if (!ctx) return DM_EINVAL;
    Choice c = choose(ctx, dm::kSketch, k, 0, 0);
    c.form = form;
    if (large_nnz >= 0) c.large_nnz = large_nnz;
    return run_sets(ctx, indptr, indices, weights, n_sets, dm::kSketch, k, 0, 0, seed, nullptr, out, nullptr, st, queue,
                    &c);
}

cudaError_t status_to_host(dm_ctx *ctx, cudaStream_t st) {
    return cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
}

int status_take(dm_ctx *ctx, cudaStream_t st) {
    const int s = *ctx->h_status;
    if (s) {
        *ctx->h_status = 0;
        cudaError_t e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DM_ECUDA;
    }
    return s;
}

int context_large_nnz(const dm_ctx *ctx) { return ctx->large_nnz; }

}  // namespace dm

namespace {

int run_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
               int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words,
               uint64_t *out_keys, cudaStream_t st, void *queue = nullptr) {
    return run_sets(ctx, indptr, indices, weights, n_sets, dm::kSketch, k, 0, b, seed, out_words, out_keys, nullptr,
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
        (e = dm::upload_poisson_table(T)) != cudaSuccess || (e = dm::upload_wide_table(T)) != cudaSuccess ||
        (e = dm::allow_max_shared_memory(device)) != cudaSuccess ||
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
    drop_graphs(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->side_ready) {
        cudaStreamDestroy(ctx->side.st);
        cudaEventDestroy(ctx->side.fork);
        cudaEventDestroy(ctx->side.join);
    }
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
    return run_sets(ctx, indptr, indices, weights, n_sets, dm::kLsh, L, K, 0, seed, nullptr, nullptr, out,
                    (cudaStream_t)stream);
}

int dm_lsh_scaled(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                  int64_t n_sets, int32_t L, int32_t K, uint64_t seed, const int32_t *scale_exp, uint32_t *out,
                  void *stream) {
    if (n_sets > 0 && !scale_exp) return DM_EINVAL;
    return run_sets(ctx, indptr, indices, weights, n_sets, dm::kLsh, L, K, 0, seed, nullptr, nullptr, out,
                    (cudaStream_t)stream, nullptr, nullptr, scale_exp);
}

int dm_weight_classes(dm_ctx *ctx, const int64_t *indptr, const float *weights, int64_t n_sets, int32_t *out,
                      int32_t *scale_out, int32_t norm_exp, void *stream) {
    if (!ctx || n_sets < 0) return DM_EINVAL;
    if (n_sets == 0) return DM_OK;
    if (!indptr || !weights || (!out && !scale_out)) return DM_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess)
        e = dm::launch_weight_classes(indptr, weights, n_sets, out, scale_out, norm_exp, ctx->sm_count,
                                      (cudaStream_t)stream);
    return cuda_fail(e);
}

int dm_bottomk(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
               int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream) {
    return run_sets(ctx, indptr, indices, weights, n_sets, dm::kBottomK, k, 0, 0, seed, nullptr, out, nullptr,
                    (cudaStream_t)stream);
}

int dm_sketch_f64(dm_ctx *ctx, const int64_t *indptr, const uint64_t *indices, const double *weights,
                  int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream) {
    if (!out && n_sets > 0) return DM_EINVAL;
    return dm_sketch_f64_bbit(ctx, indptr, indices, weights, n_sets, k, 0, seed, nullptr, out, stream);
}

int dm_sketch_f64_bbit(dm_ctx *ctx, const int64_t *indptr, const uint64_t *indices, const double *weights,
                       int64_t n_sets, int32_t k, int32_t b, uint64_t seed, uint64_t *out_words, uint64_t *out_keys,
                       void *stream) {
    if (!ctx || n_sets < 0 || k < 1 || k > 1024) return DM_EINVAL;
    if (!(b == 0 || b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32)) return DM_EINVAL;
    if (n_sets == 0) return DM_OK;
    if (!indptr || !indices || !weights || (b == 0 && !out_keys) || (b > 0 && !out_words)) return DM_EINVAL;
    uint64_t *out = out_keys;
    Range range("dm_sketch_f64");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e);
    dm::WideParams wp;
    wp.indptr = indptr;
    wp.indices = indices;
    wp.weights = weights;
    wp.n_sets = n_sets;
    wp.k = k;
    wp.t = (uint32_t)t_of_k(k);
    wp.sigma = dm::mix64(seed ^ dm::kSeedSalt);
    wp.phi0 = (double)ctx->phi0;
    wp.out = out;
    wp.out_words = b > 0 ? out_words : nullptr;
    wp.b = b;
    wp.words = b > 0 ? (int32_t)(((int64_t)k * b + 63) / 64) : 0;
    wp.status = ctx->d_status;
    wp.counters = ctx->counters;
    return cuda_fail(dm::launch_wide(wp, ctx->counters != nullptr, ctx->sm_count, (cudaStream_t)stream));
}

// The device address of a page-locked, mapped host array (null when it is not one).
const void *mapped_view(const void *h) {
    if (!h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();                       // an unregistered pointer is not an error here
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
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
    if (ctx->host_mode != 0) {
        // in place: the kernels address the host arrays through their device mapping
        const void *dip = mapped_view(indptr), *dix = mapped_view(indices), *dw = mapped_view(weights);
        void *dk = out_keys ? const_cast<void *>(mapped_view(out_keys)) : nullptr;
        void *dwd = b > 0 ? const_cast<void *>(mapped_view(out_words)) : nullptr;
        const bool ok = dip && dix && dw && (!out_keys || dk) && (b == 0 || dwd);
        if (ok) {
            Range range("dm_sketch_host");
            ctx->host_out = true;                 // bucket minima stay in shared memory
            rc = run_sketch(ctx, (const int64_t *)dip, (const uint32_t *)dix, (const float *)dw, n_sets, k, b, seed,
                            (uint64_t *)dwd, (uint64_t *)dk, st);
            ctx->host_out = false;
            if (rc) return rc;
            return cuda_fail(cudaStreamSynchronize(st));
        }
        if (ctx->host_mode == 1) return DM_EINVAL;
    }
    const int64_t words = b > 0 ? ((int64_t)k * b + 63) / 64 : 0;
    // chunks of about 1/host_chunks of the batch (at least 4,096 sets), two buffer sets in flight;
    // the first two and the last two chunks are a quarter and a half of that, so that the copy
    // in before the first kernel and the copy out after the last one stay short
    int64_t cs = (n_sets + ctx->host_chunks - 1) / ctx->host_chunks;
    if (cs < 4096) cs = 4096;
    if (cs > n_sets) cs = n_sets;
    std::vector<int64_t> bounds{0};
    if (n_sets >= 4 * cs && cs / 4 >= 4096) {
        bounds.push_back(cs / 4);
        bounds.push_back(cs / 4 + cs / 2);
        const int64_t end_mid = n_sets - cs / 2 - cs / 4, mid = end_mid - bounds.back();
        const int64_t nm = (mid + cs - 1) / cs;
        for (int64_t i = 1; i <= nm; ++i) bounds.push_back(bounds[2] + mid * i / nm);
        bounds.push_back(n_sets - cs / 4);
        bounds.push_back(n_sets);
    } else {
        for (int64_t s0 = cs; s0 < n_sets; s0 += cs) bounds.push_back(s0);
        bounds.push_back(n_sets);
    }
    int64_t max_nnz = 0;
    for (size_t i = 0; i + 1 < bounds.size(); ++i) {
        const int64_t z = indptr[bounds[i + 1]] - indptr[bounds[i]];
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
    Range range("dm_sketch_host");
    // the staged work starts after everything already queued on the caller's stream
    if ((e = cudaEventRecord(ctx->ev_start, st)) != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < 2; ++i)
        if ((e = cudaStreamWaitEvent(ctx->copy_stream[i], ctx->ev_start, 0)) != cudaSuccess) return cuda_fail(e);
    for (int chunk = 0; chunk + 1 < (int)bounds.size(); ++chunk) {
        const int64_t s0 = bounds[chunk], s1 = bounds[chunk + 1], n = s1 - s0;
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

int dm_autotune(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                int64_t n_sets, int32_t lsh, int32_t k, int32_t K_or_b, uint64_t seed, int64_t max_sets,
                dm_tuning *result, void *stream) {
    if (!ctx || lsh < 0 || lsh > 2) return DM_EINVAL;
    const int kind = lsh;                        // 0 sketches, 1 (L, K) LSH, 2 bottom-k
    int rc = check_csr(indptr, indices, weights, n_sets);
    if (rc) return rc;
    const bool is_lsh = kind == dm::kLsh;
    const int K = is_lsh ? K_or_b : 0, b = kind == dm::kSketch ? K_or_b : 0;
    if (n_sets == 0) return DM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t n = n_sets < (max_sets > 0 ? max_sets : 65536) ? n_sets : (max_sets > 0 ? max_sets : 65536);

    // the prefix's largest row decides whether the large-set threshold is worth trying
    std::vector<int64_t> ip((size_t)n + 1);
    if ((e = cudaMemcpyAsync(ip.data(), indptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e);
    int64_t max_nnz = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (ip[s + 1] < ip[s]) return DM_EINVAL;
        max_nnz = ip[s + 1] - ip[s] > max_nnz ? ip[s + 1] - ip[s] : max_nnz;
    }

    // outputs of the trial runs go to scratch (the caller's buffers are not touched)
    const int64_t words = b > 0 ? ((int64_t)k * b + 63) / 64 : 0;
    const size_t out_bytes = is_lsh ? (size_t)n * k * 4 : (b > 0 ? (size_t)n * words * 8 : (size_t)n * k * 8);
    if (is_lsh ? (k < 1 || k > 1024 || K < 1 || K > 32)
               : kind == dm::kBottomK ? (k < 1 || k > 1024 || K_or_b != 0)
                                      : (k < 1 || k > 8192 || !(b == 0 || b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32)))
        return DM_EINVAL;
    if ((rc = ensure_queue(ctx, n)) != DM_OK) return rc;
    if (ctx->budget && out_bytes + queue_bytes(ctx->queue_cap) + ctx->d_stage_bytes > ctx->budget) return DM_ENOMEM;
    void *d_out = nullptr;
    if ((e = cudaMalloc(&d_out, out_bytes)) != cudaSuccess) return cuda_fail(e);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    for (auto &x : ev)
        if ((e = cudaEventCreate(&x)) != cudaSuccess) break;

    // median of three timed runs after one warm-up; +inf if the choice is rejected
    auto time_choice = [&](const Choice &c, float &ms) -> int {
        float v[3];
        for (int r = 0; r < 4; ++r) {
            cudaError_t er = cudaEventRecord(ev[0], st);
            if (er != cudaSuccess) return cuda_fail(er);
            int q = run_sets(ctx, indptr, indices, weights, n, kind, k, K, b, seed,
                             (!is_lsh && b > 0) ? (uint64_t *)d_out : nullptr,
                             (!is_lsh && b == 0) ? (uint64_t *)d_out : nullptr,
                             is_lsh ? (uint32_t *)d_out : nullptr, st, nullptr, &c);
            if (q == DM_EINVAL) {
                ms = 3.0e38f;
                return DM_OK;
            }
            if (q) return q;
            if ((er = cudaEventRecord(ev[1], st)) != cudaSuccess || (er = cudaEventSynchronize(ev[1])) != cudaSuccess)
                return cuda_fail(er);
            if (r > 0 && (er = cudaEventElapsedTime(&v[r - 1], ev[0], ev[1])) != cudaSuccess) return cuda_fail(er);
        }
        float lo = v[0] < v[1] ? v[0] : v[1], hi = v[0] < v[1] ? v[1] : v[0];
        ms = v[2] < lo ? lo : (v[2] > hi ? hi : v[2]);
        return DM_OK;
    };

    const bool use_graph = ctx->use_graph;
    ctx->use_graph = false;                          // trials of one-off plans
    Choice best{ctx->form == 1 ? 0 : ctx->form, ctx->warps_per_block, is_lsh ? ctx->phi0_lsh : ctx->phi0,
                ctx->large_nnz, ctx->large_work, ctx->slots};
    float best_ms = 0.f, default_ms = 0.f;
    rc = e == cudaSuccess ? time_choice(best, best_ms) : cuda_fail(e);
    default_ms = best_ms;
    // coordinate search: phi0, then warps per block, then the large-set threshold, then the form
    auto try_set = [&](auto apply, const auto &values) {
        for (auto v : values) {
            if (rc) return;
            Choice c = best;
            apply(c, v);
            float ms = 0.f;
            rc = time_choice(c, ms);
            if (!rc && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    };
    if (!rc) {
        const std::vector<float> phis = is_lsh ? std::vector<float>{2.f, 3.f, 4.f, 6.f, 8.f}
                                               : std::vector<float>{1.f, 1.25f, 1.5f, 2.f};
        try_set([](Choice &c, float v) { c.phi0 = v; }, phis);
        try_set([](Choice &c, int v) { c.wpb = v; }, std::vector<int>{2, 4, 8});
        if (kind == dm::kSketch && max_nnz >= 256)
            try_set([](Choice &c, int v) { c.large_nnz = v; }, std::vector<int>{0, 256, 512, 1024, 2048, 4096, 8192});
        if (kind == dm::kSketch)
            try_set([](Choice &c, float v) { c.large_work = v; },
                    std::vector<float>{0.f, 16384.f, 32768.f, 65536.f, 131072.f});
        try_set([](Choice &c, int v) { c.form = v; }, std::vector<int>{0, 2});
        // slot storage: the bucket minima in shared memory or in the output row (sketches whose
        // trials write keys, i.e. b = 0)
        if (kind == dm::kSketch && b == 0) try_set([](Choice &c, int v) { c.slots = v; }, std::vector<int>{1, 2});
    }
    ctx->use_graph = use_graph;
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    cudaFree(d_out);
    if (rc) return rc;
    // trial runs of rows with bad weights recorded an error: report it like a call would
    if ((rc = dm_sync_status(ctx, stream)) != DM_OK) return rc;
    bool found = false;
    for (auto &t : ctx->tuned)
        if (t.kind == kind && t.k == k && t.K == K && t.b == b) {
            t.c = best;
            found = true;
        }
    if (!found) ctx->tuned.push_back(TunedEntry{kind, k, K, b, best});
    if (result) {
        result->form = best.form;
        const bool row = kind == dm::kSketch && b == 0 && best.slots != 1;
        result->warps_per_block = best.wpb > 0 ? best.wpb : auto_warps(kind, k, K, row);
        result->phi0_1024 = (int32_t)(best.phi0 * 1024.0f + 0.5f);
        result->large_nnz = best.large_nnz;
        result->large_work = (int32_t)best.large_work;
        result->sets_timed = n;
        result->ms_default = default_ms;
        result->ms_tuned = best_ms;
        result->slots = best.slots;
    }
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
    int line = 0;                                 // the checked build's index checks
    if (dm::take_check_line(&line, st) != cudaSuccess) return DM_ECUDA;
    if (line) return DM_ECHECK;
    return s;
}

int32_t dm_build_flags(void) {
#ifdef DM_CHECKED
    return 1;
#else
    return 0;
#endif
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
        case DM_EAGAIN: return "admission budget full; retry later";
        case DM_ECHECK: return "an index check of the checked build failed (a library defect)";
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
        case DM_OPT_LARGE_WORK:
            if (value < 0 || value > (1ll << 40)) return DM_EINVAL;
            ctx->large_work = (float)value;
            return DM_OK;
        case DM_OPT_HOST_CHUNKS:
            if (value < 1 || value > 256) return DM_EINVAL;
            ctx->host_chunks = (int)value;
            return DM_OK;
        case DM_OPT_HOST_MODE:
            if (value < 0 || value > 2) return DM_EINVAL;
            ctx->host_mode = (int)value;
            return DM_OK;
        case DM_OPT_SLOTS:
            if (value < 0 || value > 2) return DM_EINVAL;
            ctx->slots = (int)value;
            return DM_OK;
        case DM_OPT_LSH_PHI0:
            if (value < 1 || value > 1024 * 1024) return DM_EINVAL;
            ctx->phi0_lsh = (float)value / 1024.0f;
            return DM_OK;
        case DM_OPT_WARPS_PER_BLOCK:
            if (value < 0 || value > 8) return DM_EINVAL;   // kernels are built for <= 256 threads
            ctx->warps_per_block = (int)value;
            return DM_OK;
        case DM_OPT_GRAPH:
            if (value < 0 || value > 1) return DM_EINVAL;
            ctx->use_graph = value != 0;
            if (!ctx->use_graph) {
                cudaSetDevice(ctx->device);
                drop_graphs(ctx);
            }
            return DM_OK;
        case DM_OPT_TUNED:
            if (value < 0 || value > 2) return DM_EINVAL;
            if (value == 2) ctx->tuned.clear();              // forget every dm_autotune choice
            else ctx->use_tuned = value != 0;
            return DM_OK;
        default:
            return DM_EINVAL;
    }
}

int dm_set_tuning(dm_ctx *ctx, int32_t lsh, int32_t k, int32_t K_or_b, const dm_tuning *tuning) {
    if (!ctx || !tuning || lsh < 0 || lsh > 2 || k < 1) return DM_EINVAL;
    const dm_tuning &t = *tuning;
    if (t.form < 0 || t.form > 2 || t.warps_per_block < 0 || t.warps_per_block > 8 || t.phi0_1024 < 1 ||
        t.phi0_1024 > 1024 * 1024 || t.large_nnz < 0 || t.large_work < 0 || t.slots < 0 || t.slots > 2)
        return DM_EINVAL;
    const int kind = lsh, K = kind == dm::kLsh ? K_or_b : 0, b = kind == dm::kSketch ? K_or_b : 0;
    const Choice c{t.form, t.warps_per_block, (float)t.phi0_1024 / 1024.0f, t.large_nnz, (float)t.large_work,
                   t.slots};
    for (auto &e : ctx->tuned)
        if (e.kind == kind && e.k == k && e.K == K && e.b == b) {
            e.c = c;
            return DM_OK;
        }
    ctx->tuned.push_back(TunedEntry{kind, k, K, b, c});
    return DM_OK;
}

int64_t dm_t_of_k(int32_t k) { return t_of_k(k); }

void dm_poisson_thresholds(uint32_t *out) {
    const uint32_t *T = table();
    for (int n = 0; n < 12; ++n) out[n] = T ? T[n] : 0;
}

}  // extern "C"
