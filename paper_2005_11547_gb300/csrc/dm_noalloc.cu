// dm_sketch_noalloc: the sketch entry point for callers that cannot let the library allocate.
//
// Some host programs do not allow a library to call cudaMalloc: a framework that hands every
// byte of device memory to its own caching allocator (a raw allocation behind its back would
// fragment its pools or push it past its budget), or a process that reserved the whole device
// up front.  Such callers cannot create a dm_ctx, whose work queue, counters and status word
// live in memory the context allocates.  This entry point runs the same two kernels as
// dm_sketch with that scratch placed instead in a fixed, file-scope device array, so a call
// touches only the caller's buffers and this array.
//
// The array is sized for DM_NOALLOC_MAX_SETS sets (about 1 MiB) and exists on every GPU that
// loads the library until the process exits.  All calls share it: two calls whose work
// overlaps on a GPU (different streams, or different host threads) race on it and may give
// wrong results.  The first call on a device looks up the array's device address, loads the
// Poisson table there and raises the kernels' shared-memory limit.  Every call ends with a
// synchronisation on its stream, so no call can be captured into a CUDA graph: on a capturing
// stream the call is refused before any work.
#include <mutex>

#include "dm_device.cuh"
#include "dm_internal.h"

namespace {

constexpr int64_t kMaxSets = DM_NOALLOC_MAX_SETS;
constexpr size_t kQueueBytes = (size_t)kMaxSets * 4;
// layout: int32 queue[kMaxSets] | queue count, fast and general work counters, pad | status
constexpr size_t kScratchBytes = kQueueBytes + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool done = false;
    int rc = DM_OK;
    unsigned char *scratch = nullptr;   // device address of g_scratch on that device
    int sm_count = 0;
};

std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the device address of the scratch array (the
// host-side symbol is only a stand-in and must never be passed to a kernel), the SM count and
// the Poisson table of Algorithm 1.
int setup_device(int dev, DeviceSetup **out) {
    if (dev < 0 || dev >= kMaxDevices) return DM_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
        uint32_t T[12];
        dm_poisson_thresholds(T);
        if (e == cudaSuccess && T[0] == 0) {
            s.rc = DM_EINVAL;
        } else {
            if (e == cudaSuccess) e = dm::upload_poisson_table(T);
            if (e == cudaSuccess) e = dm::allow_max_shared_memory(dev);
            s.rc = e == cudaSuccess ? DM_OK : DM_ECUDA;
        }
        s.scratch = (unsigned char *)ptr;
        s.done = s.rc == DM_OK;          // a failed set-up is tried again by the next call
    }
    *out = &s;
    return s.rc;
}

}  // namespace

extern "C" int dm_sketch_noalloc(const int64_t *indptr, const uint32_t *indices, const float *weights,
                                 int64_t n_sets, int32_t k, uint64_t seed, uint64_t *out, void *stream) {
    if (n_sets < 0 || n_sets > kMaxSets) return DM_EINVAL;
    if (n_sets > 0 && (!indptr || !indices || !weights || !out)) return DM_EINVAL;
    if (k < 1 || k > 8192) return DM_EINVAL;
    const int64_t t = dm_t_of_k(k);
    if (t <= 0) return DM_EINVAL;
    if (n_sets == 0) return DM_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DM_ECUDA;
    DeviceSetup *ds = nullptr;
    int rc = setup_device(dev, &ds);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return DM_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return DM_EINVAL;     // the call synchronises its stream

    // warps per block: as many as fit 96 KB of shared memory, at most 8
    const bool key_row = true;                    // out is always given: minima in the output row
    const size_t wf = dm::warp_bytes(dm::kSketch, k, 0, 0, key_row), wg = dm::warp_bytes(dm::kSketch, k, 0, 1, key_row);
    int wpb = (int)((96 * 1024) / (wf > wg ? wf : wg));
    wpb = wpb > 8 ? 8 : (wpb < 1 ? 1 : wpb);

    dm::SketchParams p{};
    p.indptr = indptr;
    p.indices = indices;
    p.weights = weights;
    p.n_sets = n_sets;
    p.k = k;
    p.t = (uint32_t)t;
    p.sigma = dm::mix64(seed ^ dm::kSeedSalt);
    p.phi0 = dm::kDefaultPhi0;
    p.out_keys = out;
    p.warps_per_block = wpb;
    p.warp_bytes = (int32_t)wg;
    p.warp_bytes_fast = (int32_t)wf;
    p.sink_bytes = (int32_t)dm::sink_bytes(dm::kSketch, k, 0, key_row);
    p.key_row = key_row;
    p.queue = (int32_t *)ds->scratch;
    p.queue_count = (unsigned int *)(ds->scratch + kQueueBytes);     // count, then the work counters
    p.work_next = p.queue_count + 1;
    p.status = (int *)(ds->scratch + kQueueBytes + 16);

    const int64_t blocks = (n_sets + wpb - 1) / wpb;
    const int64_t cap0 = (int64_t)ds->sm_count * dm::blocks_per_sm(dm::kSketch, 0, false, wpb, wf * wpb, key_row);
    const int64_t cap1 = (int64_t)ds->sm_count * dm::blocks_per_sm(dm::kSketch, 1, false, wpb, wg * wpb, key_row);
    // the status word keeps the previous call's value: clear it (launch_sets clears the counters)
    cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = dm::launch_sets(p, dm::kSketch, false, false, (int)(blocks < cap0 ? blocks : cap0),
                            (int)(blocks < cap1 ? blocks : cap1), st);
    // return the first error the kernels recorded (the call is synchronous)
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, p.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DM_ENOMEM : DM_ECUDA;
    return status;
}
