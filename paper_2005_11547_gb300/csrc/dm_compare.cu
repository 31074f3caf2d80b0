// Similarity estimation from sketches (Section 1.1, "Similarity estimation"): the number of the k
// minhash slots whose values agree between two sets.  For uint64 keys the expected count is k J
// (Eq. 1); for b-bit values it is k (J + (1 - J) 2^-b).  Row-aligned pairs stream both batches
// once (HBM-bound); the cross form compares every row of one batch with every row of another,
// staging tiles of both in shared memory.
#include <cstdint>

#include "dm_internal.h"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Equal b-bit fields among the first f fields of x = a ^ c (a field is equal iff it is zero).
__device__ __forceinline__ uint32_t equal_fields(uint64_t x, int bits, uint32_t f) {
    // fold each field onto its lowest bit, then count the fields that are nonzero
    for (int s = 1; s < bits; s <<= 1) x |= x >> s;
    uint64_t low = 0;                            // bit 0 of every field
    switch (bits) {
        case 1: low = ~0ull; break;
        case 2: low = 0x5555555555555555ull; break;
        case 4: low = 0x1111111111111111ull; break;
        case 8: low = 0x0101010101010101ull; break;
        case 16: low = 0x0001000100010001ull; break;
        default: low = 0x0000000100000001ull; break;
    }
    const uint32_t per = 64u / (uint32_t)bits;
    if (f < per) low &= (1ull << (f * (uint32_t)bits)) - 1;   // fields past k are not counted
    return f - (uint32_t)__popcll(x & low);
}

// Row-aligned key pairs: a warp per pair, lanes striding the k slots.
__global__ void __launch_bounds__(256) pairs_keys(const uint64_t *a, const uint64_t *c, int64_t n, int k,
                                                  uint32_t *out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const uint64_t *ra = a + i * k, *rc = c + i * k;
        uint32_t m = 0;
        for (int j = lane; j < k; j += 32) m += ra[j] == rc[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(kFull, m, o);
        if (lane == 0) out[i] = m;
    }
}

// Row-aligned b-bit pairs: a thread per pair over its W words.
__global__ void __launch_bounds__(256) pairs_words(const uint64_t *a, const uint64_t *c, int64_t n, int k, int bits,
                                                   int W, uint32_t *out) {
    const uint32_t per = 64u / (uint32_t)bits;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t m = 0;
        for (int w = 0; w < W; ++w) {
            const uint32_t left = (uint32_t)k - (uint32_t)w * per;
            m += equal_fields(a[i * W + w] ^ c[i * W + w], bits, left < per ? left : per);
        }
        out[i] = m;
    }
}

// Cross form, keys: a block computes a 32 x 32 tile of pairs (8 per thread), the k slots taken
// in chunks of 32 staged in shared memory.
constexpr int kTile = 32, kChunk = 32;

__global__ void __launch_bounds__(128) cross_keys(const uint64_t *a, const uint64_t *c, int64_t na, int64_t nc, int k,
                                                  uint32_t *out) {
    __shared__ uint64_t sa[kTile][kChunk + 1], sc[kTile][kChunk + 1];
    const int64_t i0 = (int64_t)blockIdx.y * kTile, j0 = (int64_t)blockIdx.x * kTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;       // ty: 0..3, rows ty, ty+4, ...
    uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q0 = 0; q0 < k; q0 += kChunk) {
        for (int r = ty; r < kTile; r += 4) {
            const int q = q0 + tx;
            sa[r][tx] = (i0 + r < na && q < k) ? a[(i0 + r) * k + q] : 0ull;
            sc[r][tx] = (j0 + r < nc && q < k) ? c[(j0 + r) * k + q] : 1ull;   // never equal past k
        }
        __syncthreads();
        const int qn = k - q0 < kChunk ? k - q0 : kChunk;
        for (int q = 0; q < qn; ++q) {
            const uint64_t vc = sc[tx][q];
#pragma unroll
            for (int s = 0; s < 8; ++s) m[s] += sa[ty + 4 * s][q] == vc;
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int64_t i = i0 + ty + 4 * s, j = j0 + tx;
        if (i < na && j < nc) out[i * nc + j] = m[s];
    }
}

// Cross form, b-bit words: a thread per pair, rows of both sides staged per 32 x 32 tile.
constexpr int kMaxWords = 64;                   // k b / 64 <= 64 words per row in this form

__global__ void __launch_bounds__(128) cross_words(const uint64_t *a, const uint64_t *c, int64_t na, int64_t nc, int k,
                                                   int bits, int W, uint32_t *out) {
    extern __shared__ uint64_t sm[];
    uint64_t *sa = sm, *sc = sm + (size_t)kTile * W;
    const int64_t i0 = (int64_t)blockIdx.y * kTile, j0 = (int64_t)blockIdx.x * kTile;
    for (int e = threadIdx.x; e < kTile * W; e += blockDim.x) {
        const int r = e / W, w = e % W;
        sa[e] = i0 + r < na ? a[(i0 + r) * W + w] : 0ull;
        sc[e] = j0 + r < nc ? c[(j0 + r) * W + w] : 0ull;
    }
    __syncthreads();
    const uint32_t per = 64u / (uint32_t)bits;
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = e / kTile, s = e % kTile;
        const int64_t i = i0 + r, j = j0 + s;
        if (i >= na || j >= nc) continue;
        uint32_t m = 0;
        for (int w = 0; w < W; ++w) {
            const uint32_t left = (uint32_t)k - (uint32_t)w * per;
            m += equal_fields(sa[r * W + w] ^ sc[s * W + w], bits, left < per ? left : per);
        }
        out[i * nc + j] = m;
    }
}

// Top-k neighbours (Section 1.1: rows of c ranked by their estimated similarity to a query row
// of a, that is by agreeing slots).  A block takes 32 query rows and a span of c rows in tiles of
// 32; for each tile it computes the 32 x 32 agreeing counts exactly as the cross form does, then
// each warp folds its 8 query rows' 32 candidates into their running lists in shared memory.  A
// list entry is the 64-bit rank key (count + 1) 2^32 + (2^32 - 1 - row): a larger key is a larger
// count, or the same count and a smaller row; 0 is an empty entry.  With several spans per query
// tile, each writes its lists to a scratch array and topk_merge folds them.
constexpr int kMaxTopk = 32;

__device__ __forceinline__ uint64_t topk_key(uint32_t count, uint32_t row) {
    return ((uint64_t)(count + 1u) << 32) | (uint64_t)(0xFFFFFFFFu - row);
}

// descending bitonic sort of one value per lane
__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t v, int lane) {
    for (int size = 2; size <= 32; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t o = __shfl_xor_sync(kFull, v, stride);
            const bool desc = (lane & size) == 0;          // this lane's run of `size` descends
            const bool low = (lane & stride) == 0;
            v = (low == desc) ? (v > o ? v : o) : (v < o ? v : o);
        }
    return v;
}

// The 32 largest of two descending lists (one value per lane each), descending: the elementwise
// maximum of one list and the other reversed is a bitonic sequence holding exactly those 32, and
// a bitonic merge sorts it.
__device__ __forceinline__ uint64_t warp_top_merge(uint64_t l, uint64_t c, int lane) {
    const uint64_t cr = __shfl_sync(kFull, c, 31 - lane);
    uint64_t v = l > cr ? l : cr;
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint64_t o = __shfl_xor_sync(kFull, v, stride);
        v = (lane & stride) == 0 ? (v > o ? v : o) : (v < o ? v : o);
    }
    return v;
}

__device__ __forceinline__ void topk_write(uint64_t key, uint32_t *oidx, uint32_t *ocnt, size_t o) {
    oidx[o] = key ? 0xFFFFFFFFu - (uint32_t)key : 0xFFFFFFFFu;
    ocnt[o] = key ? (uint32_t)(key >> 32) - 1u : 0u;
}

template <bool WORDS>
__global__ void __launch_bounds__(128) topk_partial(const uint64_t *a, const uint64_t *c, int64_t na, int64_t nc,
                                                    int k, int bits, int W, int topk, int64_t span, uint64_t *part,
                                                    uint32_t *oidx, uint32_t *ocnt) {
    extern __shared__ uint64_t sm[];                                  // b-bit rows: [32][W] of a, then of c
    __shared__ uint32_t cnt[kTile][kTile + 1];
    __shared__ uint64_t best[kTile][kMaxTopk];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    const int64_t jb = (int64_t)blockIdx.y * span, je = jb + span < nc ? jb + span : nc;
    for (int e = threadIdx.x; e < kTile * kMaxTopk; e += blockDim.x) best[e / kMaxTopk][e % kMaxTopk] = 0ull;
    __syncthreads();
    for (int64_t j0 = jb; j0 < je; j0 += kTile) {
        uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};                    // rows ty + 4 s, column tx
        if constexpr (!WORDS) {
            uint64_t *sa = sm, *sc = sm + kTile * (kChunk + 1);       // [32][33] each
            for (int q0 = 0; q0 < k; q0 += kChunk) {
                for (int r = ty; r < kTile; r += 4) {
                    const int q = q0 + tx;
                    sa[r * (kChunk + 1) + tx] = (i0 + r < na && q < k) ? a[(i0 + r) * k + q] : 0ull;
                    sc[r * (kChunk + 1) + tx] = (j0 + r < je && q < k) ? c[(j0 + r) * k + q] : 1ull;
                }
                __syncthreads();
                const int qn = k - q0 < kChunk ? k - q0 : kChunk;
                for (int q = 0; q < qn; ++q) {
                    const uint64_t vc = sc[tx * (kChunk + 1) + q];
#pragma unroll
                    for (int s = 0; s < 8; ++s) m[s] += sa[(ty + 4 * s) * (kChunk + 1) + q] == vc;
                }
                __syncthreads();
            }
        } else {
            uint64_t *sa = sm, *sc = sm + (size_t)kTile * W;
            for (int e = threadIdx.x; e < kTile * W; e += blockDim.x) {
                const int r = e / W, w = e % W;
                sa[e] = i0 + r < na ? a[(i0 + r) * W + w] : 0ull;
                sc[e] = j0 + r < je ? c[(j0 + r) * W + w] : 0ull;
            }
            __syncthreads();
            const uint32_t per = 64u / (uint32_t)bits;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int r = ty + 4 * s;
                for (int w = 0; w < W; ++w) {
                    const uint32_t left = (uint32_t)k - (uint32_t)w * per;
                    m[s] += equal_fields(sa[r * W + w] ^ sc[tx * W + w], bits, left < per ? left : per);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) cnt[ty + 4 * s][tx] = m[s];
        __syncthreads();
        for (int rr = 0; rr < 8; ++rr) {                              // warp ty: query rows 8 ty ..
            const int r = 8 * ty + rr;
            const uint64_t cand = j0 + tx < je ? topk_key(cnt[r][tx], (uint32_t)(j0 + tx)) : 0ull;
            if (__any_sync(kFull, cand > best[r][topk - 1])) {
                const uint64_t l = tx < topk ? best[r][tx] : 0ull;
                const uint64_t v = warp_top_merge(l, warp_sort_desc(cand, tx), tx);
                __syncwarp();
                if (tx < topk) best[r][tx] = v;
                __syncwarp();
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < kTile * topk; e += blockDim.x) {
        const int r = e / topk, t = e % topk;
        const int64_t i = i0 + r;
        if (i >= na) continue;
        const size_t o = ((size_t)blockIdx.y * (size_t)na + (size_t)i) * (size_t)topk + (size_t)t;
        if (part) part[o] = best[r][t];
        else topk_write(best[r][t], oidx, ocnt, o);
    }
}

// A warp per query row folds the row's lists of all spans (each descending) into one.
__global__ void __launch_bounds__(256) topk_merge(const uint64_t *part, int64_t na, int spans, int topk,
                                                  uint32_t *oidx, uint32_t *ocnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < na; i += nw) {
        uint64_t best = 0ull;
        for (int s = 0; s < spans; ++s) {
            const uint64_t v = lane < topk ? part[((size_t)s * (size_t)na + (size_t)i) * (size_t)topk + lane] : 0ull;
            best = warp_top_merge(best, v, lane);
        }
        if (lane < topk) topk_write(best, oidx, ocnt, (size_t)i * (size_t)topk + lane);
    }
}

// Weighted Jaccard estimates from agreeing-slot counts (Section 1.1): p = m / k estimates J for
// keys (Eq. 1); for b-bit fields E[m] / k = J + (1 - J) 2^-b, so J is estimated by
// (p - 2^-b) / (1 - 2^-b).  binary64, IEEE-rounded division and subtraction in that order.
__global__ void __launch_bounds__(256) estimate_kernel(const uint32_t *m, int64_t n, double k, double r,
                                                       int bbit, double *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double p = __ddiv_rn((double)m[i], k);
        out[i] = bbit ? __ddiv_rn(__dsub_rn(p, r), __dsub_rn(1.0, r)) : p;
    }
}

}  // namespace

extern "C" int dm_estimate_jaccard(const uint32_t *matches, int64_t n, int32_t k, int32_t bits, double *out,
                                   void *stream) {
    if (n < 0 || k < 1 || k > 8192) return DM_EINVAL;
    if (!(bits == 0 || bits == 1 || bits == 2 || bits == 4 || bits == 8 || bits == 16 || bits == 32)) return DM_EINVAL;
    if (n == 0) return DM_OK;
    if (!matches || !out) return DM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DM_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (n + 255) / 256, cap = 8LL * (sms > 0 ? sms : 1);
    estimate_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, (cudaStream_t)stream>>>(
        matches, n, (double)k, bits ? 1.0 / (double)(1ull << bits) : 0.0, bits != 0, out);
    return cudaGetLastError() == cudaSuccess ? DM_OK : DM_ECUDA;
}

extern "C" int dm_compare(dm_ctx *ctx, const uint64_t *a, const uint64_t *c, int64_t n_a, int64_t n_c, int32_t k,
                          int32_t bits, int32_t mode, uint32_t *out, void *stream) {
    if (!ctx || n_a < 0 || n_c < 0 || k < 1 || k > 8192 || (mode != 0 && mode != 1)) return DM_EINVAL;
    if (!(bits == 0 || bits == 1 || bits == 2 || bits == 4 || bits == 8 || bits == 16 || bits == 32)) return DM_EINVAL;
    if (mode == 0 && n_a != n_c) return DM_EINVAL;
    const int64_t pairs = mode == 0 ? n_a : n_a * n_c;
    if (pairs == 0) return DM_OK;
    if (!a || !c || !out) return DM_EINVAL;
    const int W = bits ? (int)(((int64_t)k * bits + 63) / 64) : 0;
    if (mode == 1 && bits && W > kMaxWords) return DM_EINVAL;
    if (mode == 1 && (n_a > ((int64_t)65535 * kTile) || (n_c + kTile - 1) / kTile > 0x7FFFFFFF)) return DM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DM_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (mode == 0) {
        if (bits == 0) {
            const int64_t blocks = (n_a + 7) / 8;
            pairs_keys<<<(int)(blocks < 64LL * sms ? blocks : 64LL * sms), 256, 0, st>>>(a, c, n_a, k, out);
        } else {
            const int64_t blocks = (n_a + 255) / 256;
            pairs_words<<<(int)(blocks < 64LL * sms ? blocks : 64LL * sms), 256, 0, st>>>(a, c, n_a, k, bits, W, out);
        }
    } else {
        const dim3 grid((unsigned)((n_c + kTile - 1) / kTile), (unsigned)((n_a + kTile - 1) / kTile));
        if (bits == 0) {
            cross_keys<<<grid, 128, 0, st>>>(a, c, n_a, n_c, k, out);
        } else {
            const size_t smem = (size_t)2 * kTile * W * sizeof(uint64_t);
            cross_words<<<grid, 128, smem, st>>>(a, c, n_a, n_c, k, bits, W, out);
        }
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DM_OK : DM_ECUDA;
}

extern "C" int dm_compare_topk(dm_ctx *ctx, const uint64_t *a, const uint64_t *c, int64_t n_a, int64_t n_c,
                               int32_t k, int32_t bits, int32_t topk, uint32_t *out_idx, uint32_t *out_count,
                               void *stream) {
    if (!ctx || n_a < 0 || n_c < 0 || n_c > 0x7FFFFFFF || k < 1 || k > 8192 || topk < 1 || topk > kMaxTopk)
        return DM_EINVAL;
    if (!(bits == 0 || bits == 1 || bits == 2 || bits == 4 || bits == 8 || bits == 16 || bits == 32)) return DM_EINVAL;
    const int W = bits ? (int)(((int64_t)k * bits + 63) / 64) : 0;
    if (bits && W > kMaxWords) return DM_EINVAL;
    if (n_a == 0) return DM_OK;
    if (!out_idx || !out_count || (n_c > 0 && (!a || !c))) return DM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t outs = (size_t)n_a * (size_t)topk;
    if (n_c == 0) {                                 // every list empty
        if (cudaMemsetAsync(out_idx, 0xFF, outs * sizeof(uint32_t), st) != cudaSuccess ||
            cudaMemsetAsync(out_count, 0, outs * sizeof(uint32_t), st) != cudaSuccess)
            return DM_ECUDA;
        return DM_OK;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DM_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // spans of c per query tile: enough blocks to fill the GPU (4 per SM), each span at least
    // 32 tiles of c rows
    const int64_t qtiles = (n_a + kTile - 1) / kTile, ctiles = (n_c + kTile - 1) / kTile;
    if (qtiles > 0x7FFFFFFF) return DM_EINVAL;
    int64_t spans = (4LL * (sms > 0 ? sms : 1) + qtiles - 1) / qtiles;
    const int64_t max_spans = (ctiles + 31) / 32;
    if (spans > max_spans) spans = max_spans;
    if (spans > 65535) spans = 65535;
    if (spans < 1) spans = 1;
    const int64_t span = (ctiles + spans - 1) / spans * kTile;
    spans = (n_c + span - 1) / span;
    uint64_t *part = nullptr;
    if (spans > 1 && cudaMallocAsync((void **)&part, (size_t)spans * outs * sizeof(uint64_t), st) != cudaSuccess)
        return DM_ECUDA;
    const dim3 grid((unsigned)qtiles, (unsigned)spans);
    if (bits == 0)
        topk_partial<false><<<grid, 128, (size_t)2 * kTile * (kChunk + 1) * sizeof(uint64_t), st>>>(
            a, c, n_a, n_c, k, 0, 0, topk, span, part, out_idx, out_count);
    else
        topk_partial<true><<<grid, 128, (size_t)2 * kTile * W * sizeof(uint64_t), st>>>(
            a, c, n_a, n_c, k, bits, W, topk, span, part, out_idx, out_count);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && part) {
        const int64_t blocks = (n_a + 7) / 8, cap = 16LL * (sms > 0 ? sms : 1);
        topk_merge<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(part, n_a, (int)spans, topk, out_idx,
                                                                          out_count);
        e = cudaGetLastError();
    }
    if (part) cudaFreeAsync(part, st);
    return e == cudaSuccess ? DM_OK : DM_ECUDA;
}
