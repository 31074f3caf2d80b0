// Wide-range minhash sketches: binary64 weights and 64-bit element ids, for the norms of the
// paper's Table 1 (||x||_1 = 2^{+-64}, 2^{+-512}) and every row whose weights lie below 2^960
// (Section 4, "Synthetic data": 64-bit ids and double weights).
//
// The dart process is that of Section 2 and Algorithm 1 (regions (nu, rho) of 2^rho columns w
// and 2^nu rows r, X ~ Poi(1) darts per area, Theorem 1's k buckets and doubling limit), with
// three changes that let it stretch to regions nu, rho ~ 1000:
//   - area counters are two-level: region key z = M(e_i + gamma (1 + 2^16 nu + rho)), area key
//     a = M(z + gamma (1 + 2^32 w + r));
//   - the rank code is the upper 32 bits of the binary64 pattern of the rank rounded toward
//     zero, so the key is (code << 32) | (q mod 2^32);
//   - the limit theta is a binary64 value with zero low 32 bits (code(theta) << 32), doubled by
//     adding 2^20 to its code, for at most 17 passes.
// Weights of 2^960 or more, or rows whose largest weight is below 2^-990, are out of range:
// then every rank that can be kept, and every limit, is a normal binary64 number.
//
// Every test that decides which darts exist, hit x or pass the limit is exact: a weight is
// y = t x = M 2^q with a 128-bit M, and the position f of y inside its last weight region and
// the fraction G of the last rank region below theta are dyadic numbers (Dy) read at any scale
// by exact floor / ceiling.
//
// A warp sketches a set.  Lanes take the set's elements round-robin and walk their areas in
// Algorithm 1's order (nu, rho, w, r), with the step loop of the binary32 kernels: a lane with no
// dart left fetches its next area, every lane with a dart left evaluates one.  Kept darts go to
// the set's k buckets in shared memory by 64-bit atomicMin.  A retry pass enumerates only the band
// between the previous limit and the new one.
#include <cstring>

#include "dm_device.cuh"
#include "dm_internal.h"

namespace {

using namespace dm;
using u128 = unsigned __int128;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = 4;            // sets (warps) per block
constexpr int kPasses = 17;          // theta_0 2^16 at most
constexpr uint64_t kSat = ~0ull;

__constant__ uint32_t c_pois_wide[12];

// The geometry and code helpers below also compile for the host, so that their integer
// arithmetic can be exercised without a GPU.
#define DM_HD __host__ __device__

DM_HD inline int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}
DM_HD inline int wbitlen64(uint64_t x) { return x ? 64 - clz64(x) : 0; }
DM_HD inline int ctz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}
DM_HD inline int bitlen128(u128 x) {
    const uint64_t hi = (uint64_t)(x >> 64), lo = (uint64_t)x;
    return hi ? 128 - clz64(hi) : wbitlen64(lo);
}
DM_HD inline uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

DM_HD inline int bitlen_of(u128 x) { return bitlen128(x); }
DM_HD inline int bitlen_of(uint64_t x) { return wbitlen64(x); }
DM_HD inline int ctz_of(uint64_t x) { return ctz64(x); }

// A dyadic value Z 2^ez, plus 2^et when `tiny` is set.  The tiny term always lies below the
// lowest bit of Z 2^ez (et < ez), so it never carries into the integer part at any scale.
// Weight positions need a 128-bit Z; rank fractions fit a 64-bit one.
template <class T>
struct DyT {
    T Z;
    int ez, et;
    bool tiny;
};
using Dy = DyT<u128>;
using Dy64 = DyT<uint64_t>;

// floor(v 2^s), saturated at 2^64 - 1
template <class T>
DM_HD uint64_t dy_floor(const DyT<T> &v, int s) {
    constexpr int W = 8 * (int)sizeof(T);
    const int a = v.ez + s;
    uint64_t ip;
    if (v.Z == 0) {
        ip = 0;
    } else if (a >= 0) {
        if (bitlen_of(v.Z) + a > 64) return kSat;
        ip = (uint64_t)(v.Z << a);
    } else {
        const T q = -a >= W ? (T)0 : (T)(v.Z >> -a);
        if constexpr (sizeof(T) > 8) {
            if ((uint64_t)(q >> 64) != 0) return kSat;
        }
        ip = (uint64_t)q;
    }
    if (v.tiny) {
        const int b = v.et + s;
        if (b >= 0) {
            if (b >= 64) return kSat;
            const uint64_t add = 1ull << b;
            if (ip > kSat - add) return kSat;
            ip += add;
        }
    }
    return ip;
}

// Bit of weight 2^-j (j >= 1) of v.
template <class T>
DM_HD inline uint32_t dy_bit(const DyT<T> &v, int j) {
    constexpr int W = 8 * (int)sizeof(T);
    const int i = -j - v.ez;
    uint32_t b = (i >= 0 && i < W) ? (uint32_t)(v.Z >> i) & 1u : 0u;
    if (v.tiny && v.et == -j) b = 1u;
    return b;
}

// Exponent of the lowest set bit of v > 0.
template <class T>
DM_HD inline int dy_lsb(const DyT<T> &v) {
    return v.tiny ? v.et : v.ez + ctz_of(v.Z);
}

// Running floors floor(v 2^s) for s = s0, s0 + 1, ... are doubled and given the next bit; they
// saturate here (every value from 2^56 on is out of range for its use).
constexpr uint64_t kBig = 1ull << 60;
DM_HD inline uint64_t dbl(uint64_t R, uint32_t b) { return R >= kBig ? kBig : 2 * R + b; }
DM_HD inline uint64_t capped(uint64_t R) { return R >= kBig ? kBig : R; }

// Weight geometry of x > 0 (binary64 bits xb): y = t x, nu_top = floor(log2(1 + y)) (Algorithm
// 1's last weight region) and f with y = 2^nu_top - 1 + f 2^nu_top, 0 <= f < 1.
DM_HD int wide_geometry(uint64_t xb, uint32_t t, Dy &f) {
    const int ex = (int)((xb >> 52) & 0x7FF);
    const uint64_t fr = xb & ((1ull << 52) - 1);
    const uint64_t m = ex ? (fr | (1ull << 52)) : fr;
    const int q = ex ? ex - 1075 : -1074;              // x = m 2^q
    const u128 M = (u128)t * m;                         // y = M 2^q, M < 2^85
    f.tiny = false;
    f.et = 0;
    if (q >= 1) {                                       // y even: y + 1 does not carry
        const int L = bitlen128(M), nu = L + q - 1;
        f.Z = M - ((u128)1 << (L - 1));                 // f 2^nu = (M - 2^(L-1)) 2^q + 1
        f.ez = 1 - L;
        f.tiny = true;
        f.et = -nu;
        return nu;
    }
    if (q == 0) {
        const u128 S = M + 1;
        const int nu = bitlen128(S) - 1;
        f.Z = S - ((u128)1 << nu);
        f.ez = -nu;
        return nu;
    }
    if (-q >= 127) {                                    // y < 2^-42: region 0, f = y
        f.Z = M;
        f.ez = q;
        return 0;
    }
    const u128 S = M + ((u128)1 << -q);                 // (y + 1) 2^-q
    const int Ls = bitlen128(S), nu = Ls - 1 + q;
    if (nu == 0) {
        f.Z = M;
        f.ez = q;
        return 0;
    }
    f.Z = S - ((u128)1 << (Ls - 1));
    f.ez = q - nu;
    return nu;
}

// Rank geometry of a limit with code c: rho_top = max{rho : 2^rho - 1 < theta} and the fraction
// G = (theta + 1 - 2^rho_top) / 2^rho_top in (0, 1] of region rho_top below theta.
DM_HD void wide_pass_cut(uint32_t c, int &rho_top, Dy64 &G) {
    const int E = (int)(c >> 20) - 1023;
    const uint64_t Mt = (1ull << 20) | (c & 0xFFFFFu);  // theta = Mt 2^(E - 20)
    G.tiny = false;
    G.et = 0;
    if (E < 0) {                                        // theta < 1
        rho_top = 0;
        G.Z = Mt;
        G.ez = E - 20;
        return;
    }
    if (E <= 20) {                                      // theta 2^20 is an integer below 2^41
        const uint64_t th20 = Mt << E, lim = ((2ull << E) - 1) << 20;
        rho_top = E + (th20 > lim ? 1 : 0);
        G.Z = th20 + (1ull << 20) - (1ull << (20 + rho_top));
        G.ez = -20 - rho_top;
        return;
    }
    rho_top = E;                                        // 2^E <= theta < 2^(E+1) - 1
    G.Z = Mt - (1ull << 20);
    G.ez = -20;
    G.tiny = true;
    G.et = -E;
}

// Upper 32 bits of the binary64 pattern of rank = 2^rho - 1 + P 2^(rho - nu - 24), rounded
// toward zero (P = r 2^24 + u < 2^56; the rank is 0 or at least 2^-1022 in range).
DM_HD uint32_t wide_code(uint64_t P, int rho, int nu) {
    const int s = rho - nu - 24;
    if (rho == 0) {                                     // rank = P 2^s
        if (P == 0) return 0;
        const int L = wbitlen64(P), E = L - 1 + s;
        const uint64_t top = L >= 21 ? P >> (L - 21) : P << (21 - L);
        return ((uint32_t)(E + 1023) << 20) | ((uint32_t)top & 0xFFFFFu);
    }
    // rho >= 1: rank = 2^rho - 1 + B with B = P 2^s in [0, 2^rho); its exponent is rho when
    // B >= 1, else rho - 1
    const bool ge1 = s >= 0 ? P != 0 : (-s < 64 && (P >> -s) != 0);
    const int E = ge1 ? rho : rho - 1, a = 20 - E, c = s + a;
    // 21-bit significand floor(rank 2^a) = 2^(rho + a) + floor(P 2^c - 2^a)
    // c = -nu - 4 or -nu - 3 < 0
    const uint64_t T1 = -c >= 64 ? 0ull : P >> -c;                        // floor(P 2^c)
    int64_t F;
    if (a >= 0) {
        F = (int64_t)T1 - ((int64_t)1 << a);
    } else {                                            // 0 < 2^a < 1: borrow iff frac(P 2^c) < 2^a
        const uint64_t R = -c >= 64 ? P : (P & ((1ull << -c) - 1));       // frac = R 2^c
        const int ms = -s;                              // R 2^c < 2^a  <=>  R < 2^-s
        const bool borrow = ms >= 64 ? true : (ms >= 0 ? R < (1ull << ms) : R == 0);
        F = (int64_t)T1 - (borrow ? 1 : 0);
    }
    const int64_t mant = ((int64_t)1 << (rho + a)) + F;
    return ((uint32_t)(E + 1023) << 20) | ((uint32_t)mant & 0xFFFFFu);
}

// Limits of one pass: rows and regions below the previous limit are skipped (band).
struct WideCut {
    int rho_lo, rho_top;
    Dy64 G, Gp;        // of theta_p and theta_{p-1} (Gp = 0 on the first pass; Gp < 1)
    uint64_t RG0;      // floor(G 2^24)
    int lsbG;          // G 2^s is an integer iff lsbG >= -s
};

// One lane's walk over the areas of its elements (positions first, first + 32, ... < end).
// Per element, the walk keeps three running floors instead of re-deriving each region's bounds:
// RG = floor(G 2^(nu+24)) (rows and row limits of region rho_top), RP = floor(Gp 2^nu) (first row
// of the band in region rho_lo) and, in region nu_top, Fv = floor(f 2^(rho+24)) (columns and the
// last column's v limit).
struct WideWalk {
    int64_t p, end;
    uint64_t e;
    Dy f;
    int nu_top, nu, rho;
    uint64_t w, ncols, r, r0, r1, z, ctr, Q, RG, RP, Fv;
    uint32_t vtop;
    bool top;

    // next element with a positive weight; false when none is left
    DM_HD bool element(const WideParams &wp, const WideCut &cut) {
        for (; p < end; p += 32) {
            const double x = wp.weights[p];
            if (x > 0.0) {
                nu_top = wide_geometry(bits_of(x), wp.t, f);
                e = mix64(wp.sigma + kGolden * (wp.indices[p] + 1));
                nu = 0;
                rho = cut.rho_lo;
                RG = cut.RG0;
                RP = 0;
                if (nu_top == 0) Fv = capped(dy_floor(f, rho + 24));
                return true;
            }
        }
        return false;
    }
    // enter region (nu, rho) at its first area; returns 0 or DM_ERANGE
    DM_HD int region(const WideCut &cut) {
        if (nu == nu_top) {
            if (Fv >= (1ull << 56)) return DM_ERANGE;           // a column index 2^32
            vtop = (uint32_t)Fv & kUMask;
            ncols = (Fv >> 24) + 1;
        } else {
            if (rho > 32) return DM_ERANGE;
            ncols = 1ull << rho;
            vtop = kUMask;
        }
        top = rho == cut.rho_top;
        r0 = rho == cut.rho_lo ? RP : 0;
        if (top) {
            r1 = (RG >> 24) + (cut.lsbG < -nu ? 1 : 0);           // ceil(G 2^nu)
            if (r1 > (1ull << 32)) return DM_ERANGE;
            Q = RG + (cut.lsbG < -(nu + 24) ? 1 : 0);             // ceil(G 2^(nu+24))
        } else {
            if (nu > 32) return DM_ERANGE;
            r1 = 1ull << nu;
        }
        z = mix64(e + kGolden * (1ull + ((uint64_t)nu << 16) + (uint64_t)rho));
        w = 0;
        r = r0;
        ctr = z + kGolden * (1ull + r0);
        return 0;
    }
    // first area of the lane; false when it has none (err set on a range error)
    DM_HD bool start(const WideParams &wp, const WideCut &cut, int &err) {
        if (!element(wp, cut)) return false;
        err = region(cut);
        return err == 0;
    }
    // next area; false at the end of the lane's elements or on a range error
    DM_HD bool advance(const WideParams &wp, const WideCut &cut, int &err) {
        ++r;
        ctr += kGolden;
        if (r < r1) return true;
        if (++w < ncols) {
            r = r0;
            ctr = z + kGolden * (1ull + (w << 32) + r0);
            return true;
        }
        if (++rho > cut.rho_top) {
            rho = cut.rho_lo;
            if (++nu > nu_top) {
                p += 32;
                if (!element(wp, cut)) return false;
            } else {
                RG = dbl(RG, dy_bit(cut.G, nu + 24));
                RP = dbl(RP, dy_bit(cut.Gp, nu));
                if (nu == nu_top) Fv = capped(dy_floor(f, rho + 24));
            }
        } else if (nu == nu_top) {
            Fv = dbl(Fv, dy_bit(f, rho + 24));
        }
        err = region(cut);
        return err == 0;
    }
};

template <bool COUNT>
__device__ int wide_walk(const WideParams &wp, int64_t beg, int64_t end, const WideCut &cut,
                         unsigned long long *slots, int lane, unsigned long long *cnt) {
    WideWalk s;
    s.p = beg + lane;
    s.end = end;
    int err = 0;
    bool live = s.start(wp, cut, err), fresh = true;
    uint32_t nx = 0, uthr = 0, vmax = 0;
    uint64_t c = 0;
    // A lane that meets a range error stops (its walk returns false); the others finish the
    // pass, whose buckets are then discarded.
    while (__any_sync(kFull, live || nx)) {
        if (nx == 0 && live) {
            if (!fresh) live = s.advance(wp, cut, err);
            fresh = false;
            if (live) {
                c = mix64(s.ctr);
                nx = (uint32_t)poisson1((uint32_t)(c >> 32), c_pois_wide);
                if (s.top) {
                    const uint64_t rb = s.r << 24;
                    uthr = s.Q <= rb ? 0u : (uint32_t)min(s.Q - rb, (uint64_t)(1u << 24));
                } else {
                    uthr = 1u << 24;
                }
                vmax = (s.nu == s.nu_top && s.w + 1 == s.ncols) ? s.vtop : kUMask;
                if (COUNT) {
                    cnt[0]++;
                    cnt[1] += nx;
                }
            }
        }
        if (nx) {
            --nx;
            c += kGolden;
            const uint64_t d = mix64(c);
            const uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & kUMask;
            if (u < uthr && v <= vmax) {
                const uint32_t code = wide_code((s.r << 24) | u, s.rho, s.nu);
                const uint64_t q = mix64(d ^ kSlotSalt);
                const uint32_t j = fastrange32((uint32_t)(q >> 32), (uint32_t)wp.k);
                atomicMin(&slots[j], ((unsigned long long)code << 32) | (uint32_t)q);
                if (COUNT) cnt[2]++;
            }
        }
    }
    const unsigned bad = __ballot_sync(kFull, err != 0);
    return bad ? __shfl_sync(kFull, err, __ffs(bad) - 1) : 0;
}

template <bool COUNT>
__global__ void __launch_bounds__(32 * kWarps, 6) wide_kernel(WideParams wp) {
    extern __shared__ unsigned long long wide_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *slots = wide_smem + (size_t)wid * wp.k;
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    unsigned long long cnt[4] = {0, 0, 0, 0};
    for (int64_t set = (int64_t)blockIdx.x * kWarps + wid; set < wp.n_sets; set += nw) {
        const int64_t beg = wp.indptr[set], end = wp.indptr[set + 1];
        // row check and ||x||_1 (any order: it only sets the first limit)
        double l1 = 0.0, mx = 0.0;
        int bad = 0;
        for (int64_t i = beg + lane; i < end; i += 32) {
            const double x = wp.weights[i];
            if (!(x >= 0.0) || isinf(x)) bad |= 1;
            else if (x >= 0x1p960) bad |= 2;
            else {
                l1 += x;
                mx = fmax(mx, x);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            bad |= __shfl_xor_sync(kFull, bad, o);
            l1 += __shfl_xor_sync(kFull, l1, o);
            mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
        }
        int err = (bad & 1) ? DM_EINVAL : ((bad & 2) ? DM_ERANGE : 0);
        if (!err && mx > 0.0 && mx < 0x1p-990) err = DM_ERANGE;
        for (int j = lane; j < wp.k; j += 32) slots[j] = ~0ull;
        __syncwarp();
        if (!err && l1 > 0.0) {
            // first limit phi0 / ||x||_1 with the low 32 bits of its pattern cleared
            uint32_t c = (uint32_t)(bits_of(wp.phi0 / l1) >> 32);
            WideCut cut;
            cut.rho_lo = 0;
            cut.Gp = Dy64{0, 0, 0, false};
            for (int pass = 0;; ++pass) {
                if (pass == kPasses) {
                    err = DM_EOVERFLOW;
                    break;
                }
                wide_pass_cut(c, cut.rho_top, cut.G);
                cut.RG0 = capped(dy_floor(cut.G, 24));
                cut.lsbG = dy_lsb(cut.G);
                err = wide_walk<COUNT>(wp, beg, end, cut, slots, lane, cnt);
                if (COUNT && lane == 0) cnt[3]++;
                __syncwarp();
                if (err) break;
                bool empty = false;
                for (int j = lane; j < wp.k; j += 32) empty |= slots[j] == ~0ull;
                if (!__any_sync(kFull, empty)) break;
                // the next band starts where this limit ended
                const bool one = !cut.G.tiny && cut.G.ez < 0 && cut.G.ez > -64 &&
                                 cut.G.Z == (1ull << -cut.G.ez);                     // G == 1
                cut.rho_lo = one ? cut.rho_top + 1 : cut.rho_top;
                cut.Gp = one ? Dy64{0, 0, 0, false} : cut.G;
                c += 1u << 20;
            }
        }
        if (err && lane == 0) dm::set_status(wp.status, err);
        if (wp.out) {
            uint64_t *o = wp.out + set * (int64_t)wp.k;
            for (int j = lane; j < wp.k; j += 32) o[j] = err ? ~0ull : slots[j];
        }
        if (wp.out_words) {
            // b-bit values (Section 1.1): low b bits of the mixed key, slot j at bit j b
            uint64_t *ow = wp.out_words + set * (int64_t)wp.words;
            const uint32_t k = (uint32_t)wp.k, b = (uint32_t)wp.b;
            if (err) {
                for (int wd = lane; wd < wp.words; wd += 32) ow[wd] = ~0ull;
            } else if (b == 1) {
                for (uint32_t j0 = 0; j0 < k; j0 += 64) {
                    const uint32_t j1 = j0 + lane, j2 = j0 + 32 + lane;
                    const bool b1 = j1 < k && (mix64(slots[j1] ^ kBbitSalt) & 1);
                    const bool b2 = j2 < k && (mix64(slots[j2] ^ kBbitSalt) & 1);
                    const unsigned lo = __ballot_sync(kFull, b1), hi = __ballot_sync(kFull, b2);
                    if (lane == 0) ow[j0 >> 6] = (uint64_t)lo | ((uint64_t)hi << 32);
                }
            } else {
                const uint32_t g = 64u / b;                 // slots per word, 2..32
                const uint64_t mask = (1ull << b) - 1;
                for (uint32_t j0 = 0; j0 < k; j0 += 32) {
                    const uint32_t j = j0 + lane;
                    uint64_t v = j < k ? (mix64(slots[j] ^ kBbitSalt) & mask) << ((j * b) & 63) : 0ull;
                    for (uint32_t o = 1; o < g; o <<= 1) v |= __shfl_xor_sync(kFull, v, o);
                    if ((lane & (g - 1)) == 0 && j < k) ow[(j * b) >> 6] = v;
                }
            }
        }
        __syncwarp();
    }
    if (COUNT && wp.counters) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            unsigned long long v = cnt[i];
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0 && v) atomicAdd(&wp.counters[i], v);
        }
    }
}

}  // namespace

namespace dm {

cudaError_t upload_wide_table(const uint32_t *T) { return cudaMemcpyToSymbol(c_pois_wide, T, 12 * sizeof(uint32_t)); }

cudaError_t launch_wide(const WideParams &wp, bool count, int sm_count, cudaStream_t st) {
    const size_t smem = (size_t)kWarps * (size_t)wp.k * sizeof(unsigned long long);
    const int64_t need = (wp.n_sets + kWarps - 1) / kWarps, cap = (int64_t)sm_count * (count ? 8 : 16);
    const int grid = (int)(need < cap ? need : cap);
    if (count) wide_kernel<true><<<grid, 32 * kWarps, smem, st>>>(wp);
    else wide_kernel<false><<<grid, 32 * kWarps, smem, st>>>(wp);
    return cudaGetLastError();
}

}  // namespace dm
