// Internal declarations shared by the host API and the kernel launchers.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dartminhash.h"

namespace dm {

// Initial phi of Theorem 1's loop for sketches (any positive value gives the same bits; 1.25
// spares most retries at 25% more first-pass darts, measured faster on the W1 and W2 batches).
constexpr float kDefaultPhi0 = 1.25f;

// What a call computes: k minhash keys (Theorem 1), (L, K) LSH values, or a bottom-k sketch.
enum Kind : int { kSketch = 0, kLsh = 1, kBottomK = 2 };

struct SketchParams {
    const int64_t *indptr;
    const uint32_t *indices;
    const float *weights;
    int64_t n_sets;
    int32_t k;            // buckets (minhashes) per set, or L for LSH
    int32_t K;            // LSH: darts kept per bucket (0 for sketches)
    uint32_t t;           // Theorem 1: ceil(k ln k) + k; LSH: L K
    uint64_t sigma;       // seed key
    float phi0;           // initial phi of Theorem 1's loop
    const int32_t *scale; // optional per-set weight scale exponents (weight classes, Section 3)
    int32_t b;            // b-bit width (bbit mode)
    int32_t words;        // uint64 words per set in bbit mode
    uint64_t *out_keys;   // n_sets * k keys (may be null in bbit mode)
    uint64_t *out_words;  // bbit words (bbit mode only)
    uint32_t *out_lsh;    // LSH values (LSH mode only)
    int *status;          // first device-detected error
    unsigned long long *counters;   // optional work counters (4)
    int32_t warp_bytes;   // dynamic shared memory per warp (general kernel)
    int32_t warp_bytes_fast;  // dynamic shared memory per warp (fast kernel)
    int32_t sink_bytes;   // leading part of a warp's shared memory that holds the sink
    int32_t warps_per_block;
    int32_t *queue;             // sets for the general kernel (capacity n_sets)
    unsigned int *queue_count;  // number of queued sets; followed by the work counters
    unsigned int *work_next;    // = queue_count + 1: next work item of the fast / general / large kernel
    // 0: persistent warps over the sets in input order; 1: one warp per set, static (the plain
    // form); 2: batched (classified into fast, general and large sets, largest first)
    int32_t sched;
    int32_t *order;             // fast sets, then large sets, each largest first (capacity n_sets)
    uint8_t *cls;               // per set: class * 32 + descending size bin
    unsigned int *hist;         // 3 x 32 bin counts, then 3 x 32 bin cursors, then class totals
    int32_t large_nnz;          // sets with at least this many elements go to the block kernel
    float large_work;           // so do sets whose Lemma 2 work estimate reaches this (0: off)
    int32_t large_warps;        // warps per block of the large-set kernel
    int32_t key_row;            // sketches: bucket minima in out_keys, shared memory holds codes only
    // general kernel of the batched form: 0 every queued set; 1 the sets classified general
    // (queue[0, class total), runs beside the fast kernel); 2 the sets the fast kernel deferred
    // (queue[class total, queue count), after the fast kernel)
    int32_t gen_part;
};

// Shared memory per warp of the fast (mode 0) or general (mode 1) kernel, and of its sink
// (k buckets of minima, or L buckets of bottom-K candidates for LSH).
size_t warp_bytes(int kind, int k, int K, int mode, bool key_row = false);
size_t sink_bytes(int kind, int k, int K, bool key_row = false);

// Sketches that write their keys to device memory keep, by default, only a 16-bit filter per
// bucket in shared memory and their 64-bit minima in the output row (key-row layout), at any k:
// against minima in shared memory it measured 1-1.5% faster at k = 64 and 256, 7% at 512, and
// it is the layout that fits at large k.

// Resident blocks per SM of a kernel.
int blocks_per_sm(int kind, int mode, bool bbit, int warps_per_block, size_t smem, bool key_row = false);

cudaError_t upload_poisson_table(const uint32_t *T);

// Checked build only (-DDM_CHECKED): the line of the first failed index check since the last call,
// cleared on reading (0: none; the product build always reports 0).  Synchronises st.
cudaError_t take_check_line(int *line, cudaStream_t st);

// Raises the dynamic shared-memory limit of every sketch kernel to the device's opt-in maximum,
// once per device (thread-safe; the device must be current).  Must precede the first launch.
cudaError_t allow_max_shared_memory(int device);

// Plain form: zeroes the queue and work counters, then launches the fast kernel over all sets
// (one warp each, in input order) and the general kernel over the sets it queued.
cudaError_t launch_sets(const SketchParams &p, int kind, bool bbit, bool count, int grid_fast, int grid_general,
                        cudaStream_t st);

// Batched form: classification (fast / general / large, costliest first by a Lemma 2 work
// estimate), then the persistent
// fast kernel, the persistent general kernel (general sets and those the fast kernel defers)
// and, for sketches, the block-per-set kernel over large sets.  grid_large = 0: no large class.
// A second stream for the large-set kernel and the general kernel over the sets classified
// general, forked from and joined back to the call's stream with the two events (so the sequence
// stays capturable as a graph).
struct SideStream {
    cudaStream_t st;
    cudaEvent_t fork, join;
};
cudaError_t launch_batched(const SketchParams &p, int kind, bool bbit, bool count, int grid_fast,
                           int grid_general, int grid_large, cudaStream_t st, const SideStream *side = nullptr);

// Weight class of each set (Section 3): floor(log2 |x|_1) of the exact sum of the positive finite
// weights, 0 for sets without one.
cudaError_t launch_weight_classes(const int64_t *indptr, const float *weights, int64_t n_sets, int32_t *out,
                                  int32_t *scale_out, int32_t norm_exp, int sm_count, cudaStream_t st);

// Shared memory of the large-set kernel's blocks.
size_t large_block_bytes(int k, int warps, bool key_row);
int large_blocks_per_sm(bool bbit, int warps, size_t smem, bool key_row = false);

// Scratch of one call: queue, order, classes and the small header (counters, histogram).
size_t call_scratch_bytes(int64_t n_sets);
void carve_call_scratch(void *base, int64_t n_sets, SketchParams &p);

// Wide-range sketches (binary64 weights, 64-bit ids; dm_wide.cu).
struct WideParams {
    const int64_t *indptr;
    const uint64_t *indices;
    const double *weights;
    int64_t n_sets;
    int32_t k;
    uint32_t t;            // ceil(k ln k) + k
    uint64_t sigma;        // seed key
    double phi0;           // initial phi of Theorem 1's loop
    uint64_t *out;         // n_sets * k keys (may be null when out_words is set)
    uint64_t *out_words;   // optional b-bit words, n_sets * words
    int32_t b, words;      // b-bit width and words per set (0 without out_words)
    int *status;
    unsigned long long *counters;   // optional: areas, darts, kept, passes
};
cudaError_t upload_wide_table(const uint32_t *T);
cudaError_t launch_wide(const WideParams &wp, bool count, int sm_count, cudaStream_t st);

// Serving loop helpers (dm_api.cu).  serve_sketch: one dm_sketch call with the call's scratch at
// `queue` (call_scratch_bytes(n_sets) bytes), the given launch form and large-set threshold
// (-1: the context's).  status_to_host queues a
// copy of the context's status word to its pinned host copy; status_take, once the stream has
// been synchronized, returns that word and clears it on the device when it was set.
int serve_sketch(dm_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *weights,
                 int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *queue, int form, int large_nnz,
                 cudaStream_t st);
cudaError_t status_to_host(dm_ctx *ctx, cudaStream_t st);
int status_take(dm_ctx *ctx, cudaStream_t st);
int context_large_nnz(const dm_ctx *ctx);

}  // namespace dm
