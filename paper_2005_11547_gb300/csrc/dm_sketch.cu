// DartMinHash sketch kernel for sm_103a: one warp per weighted set.
//
// Per set (Theorem 1 of Christiani, arXiv 2005.11547): compute ||x||_1, set the rank limit
// theta = phi0 / ||x||_1, run DartHash (Algorithm 1) for darts of rank < theta, hash each
// kept dart to one of k buckets and keep the minimum key per bucket; while a bucket is
// empty, double theta and enumerate only the areas that reach above the previous limit.
//
// GPU mapping
//  * Elements are taken 32 at a time (a tile, one lane each).  Each lane computes its
//    element's area count for this pass in closed form; a warp scan flattens the tile's
//    areas and every lane walks a contiguous, equal share of them, so lanes stay busy no
//    matter how unequal the element weights are.
//  * Each area costs one hash (its Poisson count).  Areas with darts are appended to a
//    64-entry area ring and their darts (area slot, j) to a 512-entry dart ring in shared
//    memory; whenever 32 darts are queued the warp processes them together, one per lane,
//    so the variable Poisson counts never diverge the warp.
//  * A kept dart's key is atomically min-ed into the set's k buckets in shared memory.
#include "dm_device.cuh"
#include "dm_internal.h"

namespace dm {

__constant__ uint32_t c_pois[12];

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kAreaRing = 128;
constexpr int kDartRing = 512;
constexpr int kMaxPasses = 21;     // phi0 * 2^20 at most (Theorem 1's loop limit)

size_t sketch_warp_bytes(int k) {
    size_t b = (size_t)k * 8          // bucket minima
             + 3 * kAreaRing * 8      // area ring: hash, rank base, meta
             + 4 * 32 * 8             // tile: element hash, F, offset, count
             + 32 * 4                 // tile: nu_top
             + kDartRing * 2;         // dart ring
    return (b + 15) & ~(size_t)15;
}

struct WarpMem {
    uint64_t *slots, *ar_a, *ar_p, *ar_m, *te, *tF, *toff, *tcnt;
    int *tnu;
    uint16_t *dref;
};

__device__ __forceinline__ WarpMem carve(unsigned char *base, int k) {
    WarpMem m;
    m.slots = reinterpret_cast<uint64_t *>(base);
    m.ar_a = m.slots + k;
    m.ar_p = m.ar_a + kAreaRing;
    m.ar_m = m.ar_p + kAreaRing;
    m.te = m.ar_m + kAreaRing;
    m.tF = m.te + 32;
    m.toff = m.tF + 32;
    m.tcnt = m.toff + 32;
    m.tnu = reinterpret_cast<int *>(m.tcnt + 32);
    m.dref = reinterpret_cast<uint16_t *>(m.tnu + 32);
    return m;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan32(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// ------------------------------------------------------------------------------------------
// Dart staging.  An area record holds the area hash a, the rank base pb and meta =
// vmax | sh << 24 | (S << 23) << 32, so that dart j of the area has
//   d = mix64(a + gamma (j + 1)),  u = d >> 40,  v = (d >> 16) & (2^24 - 1),
//   rank = (pb + (u << sh)) 2^-S,  weight test v <= vmax.
// A dart reference is (area slot | j << 7).
// ------------------------------------------------------------------------------------------
struct Ring {
    uint32_t a_tail, d_tail, d_head;
};

__device__ __forceinline__ uint64_t pack_meta(uint64_t vmax, int sh, int S) {
    return vmax | ((uint64_t)sh << 24) | ((uint64_t)((uint32_t)S << 23) << 32);
}

__device__ __forceinline__ void stage_area(Ring &q, const WarpMem &m, int lane, unsigned lt_mask, int X,
                                           uint64_t a, uint64_t pb, uint64_t meta) {
    unsigned bal = __ballot_sync(kFull, X > 0);
    uint32_t aslot = (q.a_tail + __popc(bal & lt_mask)) & (kAreaRing - 1);
    if (X > 0) {
        m.ar_a[aslot] = a;
        m.ar_p[aslot] = pb;
        m.ar_m[aslot] = meta;
    }
    q.a_tail += __popc(bal);
    uint32_t xin = warp_incl_scan32((uint32_t)X, lane);
    uint32_t xtot = __shfl_sync(kFull, xin, 31);
    uint32_t at = q.d_tail + xin - (uint32_t)X;
    for (int j = 0; j < X; ++j) m.dref[(at + j) & (kDartRing - 1)] = (uint16_t)(aslot | (j << 7));
    q.d_tail += xtot;
    __syncwarp();
}

// Evaluate one queued dart; returns whether it is kept and its bucket and key.
__device__ __forceinline__ bool dart_eval(const WarpMem &m, uint32_t ref, uint32_t k, uint32_t cthr,
                                          uint32_t &slot, uint64_t &key) {
    int ai = ref & (kAreaRing - 1);
    uint64_t j = ref >> 7;
    uint64_t a = m.ar_a[ai], pb = m.ar_p[ai], meta = m.ar_m[ai];
    uint64_t d = mix64(a + kGolden * (j + 1));
    uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & kUMask;
    uint64_t P = pb + ((uint64_t)u << ((meta >> 24) & 63));
    // binary32 code of rank = P 2^-S rounded toward zero: exact u64 -> f32 conversion in
    // round-toward-zero mode, then the exponent lowered by S
    uint32_t code = P ? __float_as_uint(__ull2float_rz(P)) - (uint32_t)(meta >> 32) : 0u;
    if (v > ((uint32_t)meta & kUMask) || code >= cthr) return false;
    uint64_t qh = mix64(d ^ kSlotSalt);
    slot = fastrange32((uint32_t)(qh >> 32), k);
    key = ((uint64_t)code << 32) | (uint32_t)qh;
    return true;
}

// Process up to 64 queued darts, two per lane.
template <bool COUNT>
__device__ __forceinline__ void drain(int n, Ring &q, const WarpMem &m, int lane, uint32_t k, uint32_t cthr,
                                      unsigned long long &kept) {
    uint32_t r0 = m.dref[(q.d_head + lane) & (kDartRing - 1)];
    uint32_t r1 = m.dref[(q.d_head + 32 + lane) & (kDartRing - 1)];
    uint32_t s0 = 0, s1 = 0;
    uint64_t k0 = 0, k1 = 0;
    bool e0 = lane < n && dart_eval(m, r0, k, cthr, s0, k0);
    bool e1 = lane + 32 < n && dart_eval(m, r1, k, cthr, s1, k1);
    if (e0) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s0]), (unsigned long long)k0);
    if (e1) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s1]), (unsigned long long)k1);
    if (COUNT) kept += (unsigned long long)e0 + (unsigned long long)e1;
    q.d_head += (uint32_t)n;
    __syncwarp();
}

template <bool COUNT>
__device__ __forceinline__ void drain_ready(Ring &q, const WarpMem &m, int lane, uint32_t k, uint32_t cthr,
                                            unsigned long long &kept) {
    while (q.d_tail - q.d_head >= 64) drain<COUNT>(64, q, m, lane, k, cthr, kept);
}

// ------------------------------------------------------------------------------------------
// Element setup shared by both walks: weight geometry and element hash for one tile.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ bool element_setup(const SketchParams &p, int64_t pos, int64_t end, int &nutop,
                                              uint64_t &F, uint64_t &e) {
    nutop = -1;
    F = 0;
    e = 0;
    if (pos >= end) return true;
    nutop = weight_geometry(__float_as_uint(p.weights[pos]), p.t, F);
    if (nutop == -2) return false;
    if (nutop >= 0) e = mix64(p.sigma + kGolden * ((uint64_t)p.indices[pos] + 1));
    return true;
}

__device__ __forceinline__ uint64_t publish_tile(const WarpMem &m, int lane, int nutop, uint64_t F, uint64_t e,
                                                 uint64_t n_el) {
    uint64_t incl = warp_incl_scan(n_el, lane);
    m.te[lane] = e;
    m.tF[lane] = F;
    m.tnu[lane] = nutop;
    m.toff[lane] = incl - n_el;
    m.tcnt[lane] = n_el;
    __syncwarp();
    return __shfl_sync(kFull, incl, 31);
}

__device__ __forceinline__ int tile_element(const WarpMem &m, uint64_t idx) {
    int el = 0;                               // last element whose offset is <= idx
#pragma unroll
    for (int step = 16; step; step >>= 1) {
        int c = el + step;
        if (c < 32 && m.toff[c] <= idx) el = c;
    }
    return el;
}

// ------------------------------------------------------------------------------------------
// Fast walk for passes whose limit is below 1 (rho_top = rho_lo = 0): every region is one
// column (w = 0) of rows [rlo(nu), rhi(nu)), so an element's areas form a 1-D sequence.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t r0_hi(const PassCut &pc, int nu) { return nu ? (pc.gm1 >> (64 - nu)) + 1 : 1; }
__device__ __forceinline__ uint64_t r0_lo(const PassCut &pc, int nu) { return nu ? (pc.gfl_lo >> (64 - nu)) : 0; }

// sum_{nu=1..n} floor(G / 2^(64-nu)) = 2H - popc(H), H = floor(G / 2^(64-n))
__device__ __forceinline__ uint64_t shifted_sum(uint64_t G, int n) {
    if (n <= 0) return 0;
    uint64_t H = G >> (64 - n);
    return 2 * H - (uint64_t)__popcll(H);
}

__device__ __forceinline__ uint64_t r0_count(int nutop, const PassCut &pc) {
    return 1 + (uint64_t)nutop + shifted_sum(pc.gm1, nutop) - shifted_sum(pc.gfl_lo, nutop);
}

struct Walk0 {
    int el, nu, nutop;
    uint64_t r, rhi, e, F, ctr;
    uint32_t vmax;
};

__device__ __forceinline__ void w0_region(Walk0 &s, const PassCut &pc) {
    s.r = r0_lo(pc, s.nu);
    s.rhi = r0_hi(pc, s.nu);
    s.vmax = (s.nu == s.nutop) ? (uint32_t)(s.F >> 40) : kUMask;
    s.ctr = s.e + kGolden * ((((uint64_t)s.nu << 58) | s.r) + 1);
}

template <bool COUNT>
__device__ int pass_rho0(const SketchParams &p, int64_t beg, int64_t end, const PassCut &pc, const WarpMem &m,
                         int lane, Ring &q, unsigned long long *cnt) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t k = (uint32_t)p.k;
    for (int64_t tile = beg; tile < end; tile += 32) {
        int nutop;
        uint64_t F, e;
        bool ok = element_setup(p, tile + lane, end, nutop, F, e);
        if (__any_sync(kFull, !ok)) return DM_ERANGE;
        uint64_t total = publish_tile(m, lane, nutop, F, e, nutop >= 0 ? r0_count(nutop, pc) : 0);
        if (total == 0) continue;
        uint64_t share = (total + 31) >> 5;
        uint64_t lo = share * lane, hi = min(lo + share, total);
        Walk0 s;
        if (lo < hi) {
            s.el = tile_element(m, lo);
            s.e = m.te[s.el];
            s.F = m.tF[s.el];
            s.nutop = m.tnu[s.el];
            uint64_t li = lo - m.toff[s.el];
            for (s.nu = 0;; ++s.nu) {
                uint64_t rows = r0_hi(pc, s.nu) - r0_lo(pc, s.nu);
                if (li < rows) break;
                li -= rows;
            }
            w0_region(s, pc);
            s.r += li;
            s.ctr += kGolden * li;
        }
        for (uint64_t it = 0; it < share; ++it) {
            bool active = lo + it < hi;
            int X = 0;
            uint64_t a = 0;
            if (active) {
                a = mix64(s.ctr);
                X = poisson1((uint32_t)(a >> 32), c_pois);
                if (COUNT) { cnt[0]++; cnt[1] += X; }
            }
            stage_area(q, m, lane, lt_mask, X, a, s.r << 24, pack_meta(s.vmax, 0, s.nu + 24));
            drain_ready<COUNT>(q, m, lane, k, pc.cthr, cnt[2]);
            if (active) {
                ++s.r;
                s.ctr += kGolden;
                if (s.r == s.rhi) {
                    if (++s.nu > s.nutop) {
                        s.nu = 0;
                        do { ++s.el; } while (s.el < 32 && m.tcnt[s.el] == 0);
                        if (s.el < 32) {
                            s.e = m.te[s.el];
                            s.F = m.tF[s.el];
                            s.nutop = m.tnu[s.el];
                        }
                    }
                    if (s.el < 32) w0_region(s, pc);
                }
            }
        }
        __syncwarp();
    }
    return 0;
}

// ------------------------------------------------------------------------------------------
// General walk: regions (nu, rho), columns w and rows r.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t element_areas(int nutop, uint64_t F, const PassCut &pc) {
    uint64_t total = 0;
    for (int nu = 0; nu <= nutop; ++nu)
        for (int rho = pc.rho_lo; rho <= pc.rho_top; ++rho)
            total += cols(nu, rho, nutop, F) * (rows_hi(pc, nu, rho) - rows_lo(pc, nu, rho));
    return total;
}

struct Walk {
    int el, nu, rho, nutop;
    uint64_t w, r, ncols, rlo, rhi;
    uint64_t e, F, WT, rbase, packhi, ctr;
};

__device__ __forceinline__ void walk_region(Walk &s, const PassCut &pc) {
    s.ncols = cols(s.nu, s.rho, s.nutop, s.F);
    s.rlo = rows_lo(pc, s.nu, s.rho);
    s.rhi = rows_hi(pc, s.nu, s.rho);
    s.WT = (s.nu == s.nutop) ? (s.F >> (40 - s.rho)) : ~0ull;
    s.rbase = ((1ull << s.rho) - 1) << (62 - s.rho);
    s.packhi = ((uint64_t)s.nu << 58) | ((uint64_t)s.rho << 52);
}

__device__ __forceinline__ void walk_ctr(Walk &s) {
    s.ctr = s.e + kGolden * ((s.packhi | (s.w << s.nu) | s.r) + 1);
}

__device__ __forceinline__ void walk_load_element(Walk &s, const WarpMem &m) {
    s.e = m.te[s.el];
    s.F = m.tF[s.el];
    s.nutop = m.tnu[s.el];
}

__device__ __forceinline__ void walk_locate(Walk &s, uint64_t idx, const WarpMem &m, const PassCut &pc) {
    s.el = tile_element(m, idx);
    walk_load_element(s, m);
    uint64_t li = idx - m.toff[s.el];
    for (s.nu = 0; s.nu <= s.nutop; ++s.nu) {
        bool found = false;
        for (s.rho = pc.rho_lo; s.rho <= pc.rho_top; ++s.rho) {
            walk_region(s, pc);
            uint64_t nrows = s.rhi - s.rlo, c = s.ncols * nrows;
            if (li < c) {
                s.w = li / nrows;
                s.r = s.rlo + (li - s.w * nrows);
                found = true;
                break;
            }
            li -= c;
        }
        if (found) break;
    }
    walk_ctr(s);
}

__device__ __forceinline__ void walk_advance(Walk &s, const WarpMem &m, const PassCut &pc) {
    ++s.r;
    s.ctr += kGolden;
    if (s.r < s.rhi) return;
    ++s.w;
    if (s.w >= s.ncols) {
        s.w = 0;
        if (++s.rho > pc.rho_top) {
            s.rho = pc.rho_lo;
            if (++s.nu > s.nutop) {
                s.nu = 0;
                do { ++s.el; } while (s.el < 32 && m.tcnt[s.el] == 0);
                if (s.el >= 32) return;           // past the tile: the lane is done
                walk_load_element(s, m);
            }
        }
        walk_region(s, pc);
    }
    s.r = s.rlo;
    walk_ctr(s);
}

template <bool COUNT>
__device__ int pass_general(const SketchParams &p, int64_t beg, int64_t end, const PassCut &pc, const WarpMem &m,
                            int lane, Ring &q, unsigned long long *cnt) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t k = (uint32_t)p.k;
    for (int64_t tile = beg; tile < end; tile += 32) {
        int nutop;
        uint64_t F, e;
        bool ok = element_setup(p, tile + lane, end, nutop, F, e);
        if (__any_sync(kFull, !ok)) return DM_ERANGE;
        uint64_t total = publish_tile(m, lane, nutop, F, e, nutop >= 0 ? element_areas(nutop, F, pc) : 0);
        if (total == 0) continue;
        uint64_t share = (total + 31) >> 5;
        uint64_t lo = share * lane, hi = min(lo + share, total);
        Walk s;
        if (lo < hi) walk_locate(s, lo, m, pc);
        for (uint64_t it = 0; it < share; ++it) {
            bool active = lo + it < hi;
            int X = 0;
            uint64_t a = 0, pb = 0, meta = 0;
            if (active) {
                a = mix64(s.ctr);
                X = poisson1((uint32_t)(a >> 32), c_pois);
                uint64_t vmax = min(s.WT - (s.w << 24), (uint64_t)kUMask);
                pb = s.rbase + (s.r << (62 - s.nu));
                meta = pack_meta(vmax, 38 - s.nu, 62 - s.rho);
                if (COUNT) { cnt[0]++; cnt[1] += X; }
            }
            stage_area(q, m, lane, lt_mask, X, a, pb, meta);
            drain_ready<COUNT>(q, m, lane, k, pc.cthr, cnt[2]);
            if (active) walk_advance(s, m, pc);
        }
        __syncwarp();
    }
    return 0;
}

// MODE 0 (fast): sets are taken in order; every pass whose rank limit is below 1 runs the 1-D
// walk; a set needing a limit >= 1 is appended to the general queue and left to MODE 1.
// MODE 1 (general): sets are taken from the queue and computed from the first pass with the
// general walk.  Both give the same bits for a set (the output does not depend on the limits).
template <bool BBIT, bool COUNT, int MODE>
__global__ void __launch_bounds__(256, MODE == 0 ? 4 : 2) sketch_kernel(const SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpMem m = carve(smem + (size_t)wib * p.warp_bytes, p.k);
    const uint32_t k = (uint32_t)p.k;
    const int64_t n_work = MODE == 0 ? p.n_sets : (int64_t)*p.queue_count;
    for (int64_t wi = (int64_t)blockIdx.x * p.warps_per_block + wib; wi < n_work;
         wi += (int64_t)gridDim.x * p.warps_per_block) {
        const int64_t set = MODE == 0 ? wi : (int64_t)p.queue[wi];
        const int64_t beg = p.indptr[set], end = p.indptr[set + 1];
        // ||x||_1 and input validation
        float l1 = 0.f;
        bool bad = false;
        for (int64_t q = beg + lane; q < end; q += 32) {
            float x = p.weights[q];
            if (!(x >= 0.f) || isinf(x)) bad = true;
            else l1 += x;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) l1 += __shfl_xor_sync(kFull, l1, o);
        int err = __any_sync(kFull, bad) ? DM_EINVAL : 0;
        for (uint32_t j = lane; j < k; j += 32) m.slots[j] = ~0ull;
        __syncwarp();
        unsigned long long cnt[3] = {0, 0, 0};
        unsigned long long passes = 0;
        bool deferred = false;
        if (!err && l1 > 0.f) {
            uint32_t th = __float_as_uint(__fdiv_rn(p.phi0, l1));
            PassCut pc;
            pc.rho_lo = 0;
            pc.gfl_lo = 0;
            for (int pass = 0;; ++pass) {
                if (pass == kMaxPasses) { err = DM_EOVERFLOW; break; }
                RankCut rc;
                if (!rank_cut(th, rc)) { err = DM_ERANGE; break; }
                pc.rho_top = rc.rho_top;
                pc.gm1 = rc.gm1;
                pc.cthr = th;
                if (MODE == 0 && pc.rho_top != 0) { deferred = true; break; }
                Ring q = {0, 0, 0};
                err = MODE == 0 ? pass_rho0<COUNT>(p, beg, end, pc, m, lane, q, cnt)
                                : pass_general<COUNT>(p, beg, end, pc, m, lane, q, cnt);
                ++passes;
                if (err) break;
                if (q.d_tail != q.d_head)
                    drain<COUNT>((int)(q.d_tail - q.d_head), q, m, lane, k, pc.cthr, cnt[2]);
                bool empty = false;
                for (uint32_t j = lane; j < k; j += 32) empty |= (m.slots[j] == ~0ull);
                if (!__any_sync(kFull, empty)) break;
                // next band starts where this limit ended
                pc.rho_lo = rc.g_one ? rc.rho_top + 1 : rc.rho_top;
                pc.gfl_lo = rc.g_one ? 0 : rc.gfl;
                th = __float_as_uint(2.0f * __uint_as_float(th));
            }
        }
        if (COUNT) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                unsigned long long v = cnt[c];
#pragma unroll
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                if (lane == 0 && p.counters) atomicAdd(&p.counters[c], v);
            }
            if (lane == 0 && p.counters) atomicAdd(&p.counters[3], passes);
        }
        if (deferred) {
            if (lane == 0) p.queue[atomicAdd(p.queue_count, 1u)] = (int32_t)set;
            __syncwarp();
            continue;
        }
        if (err) {
            if (lane == 0) set_status(p.status, err);
            for (uint32_t j = lane; j < k; j += 32) m.slots[j] = ~0ull;
            __syncwarp();
        }
        // epilogue: keys and/or b-bit words
        if (p.out_keys)
            for (uint32_t j = lane; j < k; j += 32) p.out_keys[set * (int64_t)k + j] = m.slots[j];
        if (BBIT) {
            const int b = p.b;
            const uint64_t bmask = (1ull << b) - 1;
            uint64_t *ow = p.out_words + set * (int64_t)p.words;
            if (err) {
                // error rows are all ones, like the key rows
                for (int wd = lane; wd < p.words; wd += 32) ow[wd] = ~0ull;
            } else if (b == 1) {
                for (uint32_t j0 = 0; j0 < k; j0 += 64) {
                    uint32_t j1 = j0 + lane, j2 = j0 + 32 + lane;
                    bool b1 = j1 < k && (mix64(m.slots[j1] ^ kBbitSalt) & 1);
                    bool b2 = j2 < k && (mix64(m.slots[j2] ^ kBbitSalt) & 1);
                    unsigned lo = __ballot_sync(kFull, b1), hi = __ballot_sync(kFull, b2);
                    if (lane == 0) ow[j0 >> 6] = (uint64_t)lo | ((uint64_t)hi << 32);
                }
            } else {
                const int g = 64 / b;                  // slots per word, 2..32
                for (uint32_t j0 = 0; j0 < k; j0 += 32) {
                    uint32_t j = j0 + lane;
                    uint64_t v = 0;
                    if (j < k) v = (mix64(m.slots[j] ^ kBbitSalt) & bmask) << ((j * (uint32_t)b) & 63);
                    for (int o = 1; o < g; o <<= 1) v |= __shfl_xor_sync(kFull, v, o);
                    if ((lane & (g - 1)) == 0 && j < k) ow[(j * (uint32_t)b) >> 6] = v;
                }
            }
        }
        __syncwarp();
    }
}

cudaError_t upload_poisson_table(const uint32_t *T) {
    return cudaMemcpyToSymbol(c_pois, T, 12 * sizeof(uint32_t));
}

template <bool BBIT, bool COUNT, int MODE>
static cudaError_t launch_t(const SketchParams &p, int grid, cudaStream_t st) {
    size_t smem = (size_t)p.warp_bytes * p.warps_per_block;
    auto fn = sketch_kernel<BBIT, COUNT, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<grid, 32 * p.warps_per_block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const SketchParams &p, bool bbit, bool count, int grid, cudaStream_t st) {
    if (bbit) return count ? launch_t<true, true, MODE>(p, grid, st) : launch_t<true, false, MODE>(p, grid, st);
    return count ? launch_t<false, true, MODE>(p, grid, st) : launch_t<false, false, MODE>(p, grid, st);
}

cudaError_t launch_sketch(const SketchParams &p, bool bbit, bool count, int grid_fast, int grid_general,
                          cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.queue_count, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if ((e = launch_mode<0>(p, bbit, count, grid_fast, st)) != cudaSuccess) return e;
    return launch_mode<1>(p, bbit, count, grid_general, st);
}

}  // namespace dm
