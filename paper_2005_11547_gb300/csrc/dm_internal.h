// Internal declarations shared by the host API and the kernel launchers.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dartminhash.h"

namespace dm {

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
    int32_t *queue;             // sets deferred to the general kernel (capacity n_sets)
    unsigned int *queue_count;  // number of queued sets; followed by the two work counters
    unsigned int *work_next;    // = queue_count + 1: next work item of the fast / general kernel
};

// Shared memory per warp of the fast (mode 0) or general (mode 1) kernel, and of its sink
// (k buckets of minima, or L buckets of bottom-K candidates for LSH).
size_t warp_bytes(bool lsh, int k, int K, int mode);
size_t sink_bytes(bool lsh, int k, int K);

// Resident blocks per SM of a kernel.
int blocks_per_sm(bool lsh, int mode, bool bbit, int warps_per_block, size_t smem);

cudaError_t upload_poisson_table(const uint32_t *T);

// Zeroes the queue and work counters, then launches the fast kernel over all sets and the
// general kernel over the sets it queued, all on stream st.
cudaError_t launch_sets(const SketchParams &p, bool lsh, bool bbit, bool count, int grid_fast, int grid_general,
                        cudaStream_t st);

}  // namespace dm
