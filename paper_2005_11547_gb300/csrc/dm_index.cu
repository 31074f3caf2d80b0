// LSH tables for approximate near neighbor search (Section 1.2, "Fast similarity search";
// Section 3): L hash tables, table l keyed by the l-th (L, K) LSH value of each point.  A query
// returns the distinct points that share a value with it in at least one table.
//
// Table l is an open-addressing array of 2^h >= 2 * capacity slots, each holding a key (the value
// with an occupancy bit) and the head of a chain of nodes; node p L + l records point p's id and
// the next node of the chain.  Insertion claims or finds the value's slot with a 64-bit
// compare-and-swap and pushes its node with an atomic exchange.  A query takes a warp: lanes probe
// the tables, walk the chains into a shared-memory buffer, and the warp sorts the buffer and
// drops repeated ids (a point colliding in several tables).
#include <new>

#include "dm_device.cuh"
#include "dm_internal.h"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kQueryBuf = 2048;        // raw candidates a query may gather
constexpr int kQueryWarps = 2;         // 2 x 16 KB of candidate buffers per block
constexpr int kMaxProbes = 1 << 16;    // the tables are at most half full: probes end far sooner

__device__ __forceinline__ uint32_t slot_of(uint32_t v, int l, uint32_t mask) {
    return (uint32_t)(dm::mix64(((uint64_t)l << 32) | v) >> 32) & mask;
}

__global__ void __launch_bounds__(256) insert_kernel(const uint32_t *values, const int64_t *ids, int64_t n,
                                                     int64_t base, int L, uint32_t mask,
                                                     unsigned long long *keys, int32_t *heads, int64_t *node_id,
                                                     int32_t *node_next, int *status) {
    const int64_t total = n * L, stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t H = (uint64_t)mask + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t p = e / L;
        const int l = (int)(e - p * L);
        const uint32_t v = values[e];
        const unsigned long long key = (1ull << 32) | v;
        unsigned long long *tk = keys + (uint64_t)l * H;
        uint32_t h = slot_of(v, l, mask);
        int probes = 0;
        for (;; h = (h + 1) & mask) {
            if (++probes > kMaxProbes) {
                dm::set_status(status, DM_EOVERFLOW);
                h = 0xFFFFFFFFu;
                break;
            }
            const unsigned long long k = tk[h];
            if (k == key) break;
            if (k == 0ull) {
                const unsigned long long old = atomicCAS(tk + h, 0ull, key);
                if (old == 0ull || old == key) break;
            }
        }
        if (h == 0xFFFFFFFFu) continue;
        const int32_t node = (int32_t)((base + p) * L + l);
        node_id[node] = ids ? ids[p] : base + p;
        node_next[node] = atomicExch(heads + (uint64_t)l * H + h, node);
    }
}

__global__ void __launch_bounds__(32 * kQueryWarps) query_kernel(const uint32_t *queries, int64_t m, int L,
                                                                  uint32_t mask, const unsigned long long *keys,
                                                                  const int32_t *heads, const int64_t *node_id,
                                                                  const int32_t *node_next, int max_candidates,
                                                                  int32_t *counts, int64_t *out) {
    __shared__ int64_t buf[kQueryWarps][kQueryBuf];
    __shared__ unsigned int fill[kQueryWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t *cand = buf[wid];
    const uint64_t H = (uint64_t)mask + 1;
    const int64_t nw = (int64_t)gridDim.x * kQueryWarps;
    for (int64_t q = (int64_t)blockIdx.x * kQueryWarps + wid; q < m; q += nw) {
        if (lane == 0) fill[wid] = 0;
        __syncwarp();
        for (int l = lane; l < L; l += 32) {
            const uint32_t v = queries[q * L + l];
            const unsigned long long key = (1ull << 32) | v;
            const unsigned long long *tk = keys + (uint64_t)l * H;
            uint32_t h = slot_of(v, l, mask);
            int32_t node = -1;
            for (int probes = 0; probes < kMaxProbes; ++probes, h = (h + 1) & mask) {
                const unsigned long long k = tk[h];
                if (k == key) {
                    node = heads[(uint64_t)l * H + h];
                    break;
                }
                if (k == 0ull) break;
            }
            for (; node >= 0; node = node_next[node]) {
                const unsigned int pos = atomicAdd(&fill[wid], 1u);
                if (pos < (unsigned int)kQueryBuf) cand[pos] = node_id[node];
                else break;                              // overflowing: the count alone matters now
            }
        }
        __syncwarp();
        const unsigned int raw = fill[wid];
        int64_t *o = out + q * (int64_t)max_candidates;
        if (raw > (unsigned int)kQueryBuf) {             // more raw candidates than the buffer holds
            for (int j = lane; j < max_candidates; j += 32) o[j] = -1;
            if (lane == 0) counts[q] = -1;
            __syncwarp();
            continue;
        }
        uint32_t n2 = 32;
        while (n2 < raw) n2 <<= 1;
        for (uint32_t j = raw + lane; j < n2; j += 32) cand[j] = INT64_MAX;
        __syncwarp();
        dm::warp_bitonic_sort(cand, n2, lane);
        // distinct ids: a sorted entry is new when it differs from its predecessor
        unsigned int distinct = 0;
        for (uint32_t j0 = 0; j0 < raw; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool fresh = j < raw && (j == 0 || cand[j] != cand[j - 1]);
            const unsigned b = __ballot_sync(kFull, fresh);
            const unsigned int rank = distinct + __popc(b & ((1u << lane) - 1u));
            if (fresh && rank < (unsigned int)max_candidates) o[rank] = cand[j];
            distinct += __popc(b);
        }
        for (int j = (int)distinct + lane; j < max_candidates; j += 32) o[j] = -1;
        if (lane == 0) counts[q] = (int32_t)distinct;
        __syncwarp();
    }
}

}  // namespace

struct dm_lsh_index {
    int device = 0;
    int32_t L = 0;
    int64_t capacity = 0, n = 0;
    uint32_t mask = 0;
    unsigned long long *keys = nullptr;
    int32_t *heads = nullptr;
    int64_t *node_id = nullptr;
    int32_t *node_next = nullptr;
    int *status = nullptr;
    int sm_count = 0;
};

extern "C" {

int dm_lsh_index_destroy(dm_lsh_index *ix) {
    if (!ix) return DM_OK;
    cudaSetDevice(ix->device);
    cudaFree(ix->keys);
    cudaFree(ix->heads);
    cudaFree(ix->node_id);
    cudaFree(ix->node_next);
    cudaFree(ix->status);
    delete ix;
    return DM_OK;
}

int dm_lsh_index_create(dm_lsh_index **out, int device, int32_t L, int64_t capacity) {
    if (!out || L < 1 || L > 1024 || capacity < 1 || capacity * (int64_t)L > 0x7FFFFFFF) return DM_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return DM_EINVAL;
    dm_lsh_index *ix = new (std::nothrow) dm_lsh_index();
    if (!ix) return DM_ENOMEM;
    ix->device = device;
    ix->L = L;
    ix->capacity = capacity;
    uint64_t H = 64;
    while (H < 2 * (uint64_t)capacity) H <<= 1;
    ix->mask = (uint32_t)(H - 1);
    cudaDeviceGetAttribute(&ix->sm_count, cudaDevAttrMultiProcessorCount, device);
    const size_t slots = (size_t)L * H, nodes = (size_t)capacity * L;
    cudaError_t e;
    if ((e = cudaMalloc(&ix->keys, slots * 8)) != cudaSuccess || (e = cudaMalloc(&ix->heads, slots * 4)) != cudaSuccess ||
        (e = cudaMalloc(&ix->node_id, nodes * 8)) != cudaSuccess ||
        (e = cudaMalloc(&ix->node_next, nodes * 4)) != cudaSuccess || (e = cudaMalloc(&ix->status, 4)) != cudaSuccess ||
        (e = cudaMemset(ix->keys, 0, slots * 8)) != cudaSuccess ||
        (e = cudaMemset(ix->heads, 0xFF, slots * 4)) != cudaSuccess || (e = cudaMemset(ix->status, 0, 4)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        dm_lsh_index_destroy(ix);
        return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
    }
    *out = ix;
    return DM_OK;
}

int dm_lsh_index_insert(dm_lsh_index *ix, const uint32_t *values, const int64_t *ids, int64_t n, void *stream) {
    if (!ix || n < 0) return DM_EINVAL;
    if (n == 0) return DM_OK;
    if (!values) return DM_EINVAL;
    if (ix->n + n > ix->capacity) return DM_ENOMEM;
    if (cudaSetDevice(ix->device) != cudaSuccess) return DM_ECUDA;
    const int64_t total = n * ix->L, blocks = (total + 255) / 256, cap = 32LL * ix->sm_count;
    insert_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, (cudaStream_t)stream>>>(
        values, ids, n, ix->n, ix->L, ix->mask, ix->keys, ix->heads, ix->node_id, ix->node_next, ix->status);
    if (cudaGetLastError() != cudaSuccess) return DM_ECUDA;
    ix->n += n;
    return DM_OK;
}

int dm_lsh_index_query(dm_lsh_index *ix, const uint32_t *queries, int64_t m, int32_t max_candidates,
                       int32_t *counts, int64_t *out_ids, void *stream) {
    if (!ix || m < 0 || max_candidates < 1 || max_candidates > kQueryBuf) return DM_EINVAL;
    if (m == 0) return DM_OK;
    if (!queries || !counts || !out_ids) return DM_EINVAL;
    if (cudaSetDevice(ix->device) != cudaSuccess) return DM_ECUDA;
    const int64_t blocks = (m + kQueryWarps - 1) / kQueryWarps, cap = 16LL * ix->sm_count;
    query_kernel<<<(int)(blocks < cap ? blocks : cap), 32 * kQueryWarps, 0, (cudaStream_t)stream>>>(
        queries, m, ix->L, ix->mask, ix->keys, ix->heads, ix->node_id, ix->node_next, max_candidates, counts, out_ids);
    return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ECUDA;
}

int dm_lsh_index_size(dm_lsh_index *ix, int64_t *n) {
    if (!ix || !n) return DM_EINVAL;
    *n = ix->n;
    return DM_OK;
}

int dm_lsh_index_status(dm_lsh_index *ix, void *stream) {
    if (!ix) return DM_EINVAL;
    if (cudaSetDevice(ix->device) != cudaSuccess) return DM_ECUDA;
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, ix->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DM_ECUDA;
    if (h && (cudaMemsetAsync(ix->status, 0, 4, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess))
        return DM_ECUDA;
    return h;
}

}  // extern "C"
