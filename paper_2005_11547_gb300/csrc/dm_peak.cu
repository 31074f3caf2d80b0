// Integer-issue ceiling of the hash the method runs on: every thread chains SplitMix64's output
// function over four independent states, so the kernel is nothing but the mixer's 64-bit
// multiplies, shifts and xors.  Its rate, times the mixer's int32 operation count, is the
// measured counterpart of the nominal peak (SMs x 128 int32 lanes x clock) that the kernels'
// work is compared against.
#include "dm_device.cuh"
#include "dm_internal.h"

namespace {

__global__ void __launch_bounds__(256) mix_burn_kernel(uint64_t seed, int32_t iters, uint64_t *out) {
    const uint64_t id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t a = seed + id, b = a ^ 0x1111111111111111ull, c = a ^ 0x2222222222222222ull,
             d = a ^ 0x3333333333333333ull;
    for (int32_t i = 0; i < iters; ++i) {
        a = dm::mix64(a);
        b = dm::mix64(b);
        c = dm::mix64(c);
        d = dm::mix64(d);
    }
    out[id] = a ^ b ^ c ^ d;
}

}  // namespace

extern "C" int dm_mix64_burn(int64_t blocks, int32_t iters, uint64_t seed, uint64_t *out, void *stream) {
    if (blocks < 1 || blocks > (1 << 30) || iters < 1 || !out) return DM_EINVAL;
    mix_burn_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(seed, iters, out);
    return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ECUDA;
}
