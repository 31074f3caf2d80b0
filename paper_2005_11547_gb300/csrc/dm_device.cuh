// Device-side building blocks of the DartMinHash hot path (sm_103a).
//
// Notation follows the paper (Christiani, arXiv 2005.11547, Section 2, Algorithm 1):
// element i with weight x_i, scaled weight y = t x_i; region (nu, rho) covers scaled weights
// [2^nu - 1, 2^(nu+1) - 1) and ranks [2^rho - 1, 2^(rho+1) - 1) and is split into 2^rho
// columns w and 2^nu rows r; every area holds X ~ Poi(1) darts.  All comparisons that decide
// which darts exist, hit x or pass the rank limit are exact integer arithmetic.
#pragma once
#include <cstdint>

namespace dm {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;   // SplitMix64 increment
constexpr uint64_t kSeedSalt = 0x243F6A8885A308D3ull;
constexpr uint64_t kSlotSalt = 0x13198A2E03707344ull;
constexpr uint64_t kBbitSalt = 0xA4093822299F31D0ull;
constexpr uint64_t kLshInit = 0x082EFA98EC4E6C89ull;
constexpr int kMaxRegion = 38;        // nu, rho <= 38 keeps every fixed-point value in 64 bits
constexpr uint32_t kUMask = 0xFFFFFFu; // 24-bit uniforms U, V

// SplitMix64's output function (Steele, Lea, Flood 2014), used as a counter-based hash.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) { return s >= 64 ? 0ull : (x >> s); }
__device__ __forceinline__ int bitlen64(uint64_t x) { return 64 - __clzll((long long)x); }

// Per-element weight geometry.  Returns nu_top = floor(log2(1 + t x)) (the last weight
// region, Algorithm 1's nu bound) and F = floor(f 2^64) where f in [0, 1) is the position of
// y = t x inside region nu_top:  y = 2^nu_top - 1 + f 2^nu_top.  Returns -1 for x == 0 and -2
// when nu_top would exceed kMaxRegion.  x must be finite and >= 0.  escale: the weight counts as
// x 2^escale (the exact normalisation of a weight class, Section 3).
__device__ __forceinline__ int weight_geometry(uint32_t xbits, uint32_t t, uint64_t &F, int escale = 0) {
    uint32_t ex = (xbits >> 23) & 0xFFu, fr = xbits & 0x7FFFFFu;
    if (ex == 0 && fr == 0) return -1;
    uint64_t M = ex ? (uint64_t)(fr | 0x800000u) : (uint64_t)fr;
    int E = (ex ? (int)ex - 150 : -149) + escale;  // x 2^escale = M 2^E exactly
    if (E > 64) return -2;                          // y >= 2^64 (and keeps the shifts below defined)
    uint64_t Z = (uint64_t)t * M;                  // y = Z 2^E, Z < 2^41
    if (E >= 0) {
        if (bitlen64(Z) + E > kMaxRegion + 1) return -2;     // y >= 2^39
        uint64_t A = (Z << E) + 1;                           // y + 1 (integer)
        int nu = bitlen64(A) - 1;
        if (nu > kMaxRegion) return -2;
        F = (A - (1ull << nu)) << (64 - nu);                 // nu >= 1 here
        return nu;
    }
    int s = -E;
    if (s <= 62) {
        uint64_t A = Z + (1ull << s);                        // (y + 1) 2^s
        int L1 = bitlen64(A) - 1;                            // = nu + s
        int nu = L1 - s;
        if (nu > kMaxRegion) return -2;
        F = (A - (1ull << L1)) << (64 - L1);                 // L1 >= s >= 1
        return nu;
    }
    // y < 2^-21: region 0, f = y
    F = (s >= 64) ? shr64(Z, s - 64) : (Z << (64 - s));
    return 0;
}

// Rank geometry of a limit theta (a positive binary32): rho_top = max{rho : 2^rho - 1 < theta}
// and g = (theta + 1 - 2^rho_top) / 2^rho_top in (0, 1], the fraction of region rho_top below
// the limit, as gm1 = ceil(g 2^64) - 1 and gfl = floor(g 2^64) (gfl meaningless if g == 1).
struct RankCut {
    int rho_top;
    bool g_one;
    uint64_t gm1, gfl;
};

__device__ __forceinline__ bool rank_cut(uint32_t thbits, RankCut &c) {
    uint32_t ex = (thbits >> 23) & 0xFFu, fr = thbits & 0x7FFFFFu;
    if (ex == 0xFFu || (ex == 0 && fr == 0) || (thbits >> 31)) return false;
    uint64_t m = ex ? (uint64_t)(fr | 0x800000u) : (uint64_t)fr;
    int e = ex ? (int)ex - 150 : -149;              // theta = m 2^e
    c.g_one = false;
    if (e <= -24) {                                  // theta < 1: rho_top = 0, g = theta
        c.rho_top = 0;
        int s = e + 64;
        if (s >= 0) {
            c.gfl = m << s;
            c.gm1 = c.gfl - 1;
        } else {
            int rs = -s;
            c.gfl = shr64(m, rs);
            bool exact = rs < 64 ? ((m & ((1ull << rs) - 1)) == 0) : false;
            c.gm1 = exact ? c.gfl - 1 : c.gfl;
        }
        return true;
    }
    if (e > 15) return false;                        // theta >= 2^39
    uint64_t A = (m << (e + 23)) + (1ull << 23);     // (theta + 1) 2^23
    int L = bitlen64(A);
    int rho = ((A & (A - 1)) == 0) ? L - 25 : L - 24;
    if (rho > kMaxRegion) return false;
    uint64_t D = A - (1ull << (rho + 23));           // g 2^(rho + 23), in (0, 2^(rho+23)]
    c.rho_top = rho;
    if (D == (1ull << (rho + 23))) {
        c.g_one = true;
        c.gm1 = ~0ull;
        c.gfl = 0;
    } else {
        c.gfl = D << (41 - rho);
        c.gm1 = c.gfl - 1;
    }
    return true;
}

// Rank limits of one pass: darts with rank < theta_p are kept; areas lying wholly below the
// previous pass's limit theta_{p-1} were already processed and are skipped (band).
struct PassCut {
    int rho_lo, rho_top;
    uint64_t gm1;      // of theta_p
    uint64_t gfl_lo;   // of theta_{p-1} (0 on the first pass)
    uint32_t cthr;     // bits(theta_p): kept iff code(rank) < cthr
    uint32_t cthr_lo;  // bits(theta_{p-1}) (0 on the first pass): darts below it were seen before
};

// Rows [rlo, rhi) of region (nu, rho) that the pass visits.
__device__ __forceinline__ uint64_t rows_hi(const PassCut &pc, int nu, int rho) {
    if (rho != pc.rho_top) return 1ull << nu;
    return nu == 0 ? 1ull : (pc.gm1 >> (64 - nu)) + 1;      // ceil(g 2^nu)
}
__device__ __forceinline__ uint64_t rows_lo(const PassCut &pc, int nu, int rho) {
    if (rho != pc.rho_lo) return 0;
    return nu == 0 ? 0ull : (pc.gfl_lo >> (64 - nu));        // floor(g_prev 2^nu)
}
// Columns [0, ncols) of region (nu, rho) with lower edge <= y.
__device__ __forceinline__ uint64_t cols(int nu, int rho, int nutop, uint64_t F) {
    if (nu != nutop) return 1ull << rho;
    return rho == 0 ? 1ull : (F >> (64 - rho)) + 1;          // floor(f 2^rho) + 1
}

__device__ __forceinline__ uint32_t fastrange32(uint32_t h, uint32_t n) {
    return (uint32_t)(((uint64_t)h * n) >> 32);
}

__device__ __forceinline__ int poisson1(uint32_t u, const uint32_t *T) {
    // X = #{n : u >= T[n]}; T increasing, so stop at the first miss
    int x = (u >= T[0]) + (u >= T[1]) + (u >= T[2]) + (u >= T[3]);
    if (u >= T[4]) {
        x = 5;
        while (x < 12 && u >= T[x]) ++x;
    }
    return x;
}

// Ascending bitonic sort of n (a power of two) 64-bit keys in shared memory by one warp.
template <class T>
__device__ inline void warp_bitonic_sort(T *a, uint32_t n, int lane) {
    for (uint32_t size = 2; size <= n; size <<= 1) {
        for (uint32_t stride = size >> 1; stride; stride >>= 1) {
            for (uint32_t i = (uint32_t)lane; i < n / 2; i += 32) {
                const uint32_t lo = ((i & ~(stride - 1)) << 1) | (i & (stride - 1)), hi = lo + stride;
                const T x = a[lo], y = a[hi];
                if ((x > y) == ((lo & size) == 0)) {
                    a[lo] = y;
                    a[hi] = x;
                }
            }
            __syncwarp();
        }
    }
}

// Minimum of a 64-bit word in shared memory (saddr: its shared-space address).  A plain read
// comes first, since most candidates lose against the current minimum; otherwise a
// compare-and-swap retries until the word is at most v.  Each failed swap means another thread
// lowered the word, so the loop ends after at most as many rounds as there are concurrent
// writers.  Explicit shared-space instructions keep the address inside the block's window.
__device__ __forceinline__ void shared_min_u64(uint32_t saddr, uint64_t v) {
    uint64_t old;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(old) : "r"(saddr) : "memory");
    while (v < old) {
        uint64_t prev;
        asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(prev) : "r"(saddr), "l"(old), "l"(v) : "memory");
        if (prev == old) break;
        old = prev;
    }
}

// Atomic minimum of a 32-bit word in shared memory (saddr: its shared-space address); returns the
// previous value.
__device__ __forceinline__ uint32_t shared_min_u32(uint32_t saddr, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared.min.u32 %0, [%1], %2;" : "=r"(old) : "r"(saddr), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Index checks of the checked build (compiled with -DDM_CHECKED; the product build compiles them
// out).  DM_EXPECT(cond) is true when cond holds; when it does not, the source line of the first
// failed check is recorded in g_dm_check (read and cleared by dm_sync_status, which then returns
// DM_ECHECK) and the caller skips the access it guards.
#ifdef DM_CHECKED
static __device__ int g_dm_check = 0;             // per translation unit; the sketch kernels' is read
__device__ __forceinline__ bool dm_expect(bool ok, int line) {
    if (!ok) atomicCAS(&g_dm_check, 0, line);
    return ok;
}
#define DM_EXPECT(cond) ::dm::dm_expect((cond), __LINE__)
#else
#define DM_EXPECT(cond) true
#endif

}  // namespace dm
