// DartMinHash sketch kernel for sm_103a: one warp per weighted set.
//
// Per set (Theorem 1 of Christiani, arXiv 2005.11547): compute ||x||_1, set the rank limit
// theta = phi0 / ||x||_1, run DartHash (Algorithm 1) for darts of rank < theta, hash each
// kept dart to one of k buckets and keep the minimum key per bucket; while a bucket is
// empty, double theta and enumerate only the areas that reach above the previous limit.
//
// GPU mapping
//  * Persistent warps claim sets from a global counter, so a set that needs a second pass
//    never holds idle warps of its block.
//  * Elements are taken 32 at a time (a tile, one lane each).  Each lane computes its
//    element's area count for this pass in closed form; a warp scan flattens the tile's
//    areas and every lane walks a contiguous, equal share of them, so lanes stay busy no
//    matter how unequal the element weights are.
//  * Each area costs one hash (its Poisson count X).  A lane then emits the area's darts one
//    per iteration into a 128-entry shared-memory dart queue (position = rank of the lane
//    in a ballot), and whenever 32 or more darts are queued the warp evaluates them
//    together, so the variable Poisson counts never diverge the warp.
//  * A kept dart's key is atomically min-ed into the set's k buckets in shared memory.
#include "dm_device.cuh"
#include "dm_internal.h"

namespace dm {

__constant__ uint32_t c_pois[12];

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kQueue = 128;        // dart records per warp
constexpr int kMaxPasses = 21;     // phi0 * 2^20 at most (Theorem 1's loop limit)
constexpr int kDefer = -1;         // a pass the fast kernel leaves to the general kernel

size_t sketch_warp_bytes(int k) {
    size_t b = (size_t)k * 8          // bucket minima
             + 2 * kQueue * 8         // dart queue: dart counter, rank base | vmax
             + 3 * 32 * 8             // tile: element hash, F, offset
             + 32 * 4                 // tile: nu_top
             + kQueue * 2;            // dart queue: shift and scale of the rank
    return (b + 15) & ~(size_t)15;
}

struct WarpMem {
    uint64_t *slots, *dq_c, *dq_p, *te, *tF, *toff;
    int *tnu;
    uint16_t *dq_m;
};

__device__ __forceinline__ WarpMem carve(unsigned char *base, int k) {
    WarpMem m;
    m.slots = reinterpret_cast<uint64_t *>(base);
    m.dq_c = m.slots + k;
    m.dq_p = m.dq_c + kQueue;
    m.te = m.dq_p + kQueue;
    m.tF = m.te + 32;
    m.toff = m.tF + 32;
    m.tnu = reinterpret_cast<int *>(m.toff + 32);
    m.dq_m = reinterpret_cast<uint16_t *>(m.tnu + 32);
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

// ------------------------------------------------------------------------------------------
// Dart queue.  A record holds the dart counter c = a + gamma (j + 1) of dart j of area a,
// pv = pb | vmax (the rank base pb is a multiple of 2^24, so its low 24 bits carry the weight
// threshold) and meta = sh | S << 6, so that the dart has
//   d = mix64(c),  u = d >> 40,  v = (d >> 16) & (2^24 - 1),
//   rank = (pb + (u << sh)) 2^-S,  weight test v <= vmax.
// ------------------------------------------------------------------------------------------
struct Queue {
    uint32_t tail, head;
};

__device__ __forceinline__ uint32_t pack_meta(int sh, int S) { return (uint32_t)sh | ((uint32_t)S << 6); }

// Evaluate one queued dart; returns whether it is kept, with its bucket and key.  RHO0: every
// queued dart has rank shift sh = 0 (rank region 0), so P = pb | u.
template <bool RHO0>
__device__ __forceinline__ bool dart_eval(const WarpMem &m, uint32_t pos, uint32_t k, uint32_t cthr,
                                          uint32_t &slot, uint64_t &key) {
    const uint32_t i = pos & (kQueue - 1);
    const uint64_t pv = m.dq_p[i];
    const uint32_t meta = m.dq_m[i];
    const uint64_t d = mix64(m.dq_c[i]);
    const uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & kUMask;
    const uint64_t P = RHO0 ? ((pv & ~(uint64_t)kUMask) | u)
                            : (pv & ~(uint64_t)kUMask) + ((uint64_t)u << (meta & 63));
    // binary32 code of rank = P 2^-S rounded toward zero: exact u64 -> f32 conversion in
    // round-toward-zero mode, then the exponent lowered by S
    const uint32_t code = P ? __float_as_uint(__ull2float_rz(P)) - ((meta >> 6) << 23) : 0u;
    if (v > ((uint32_t)pv & kUMask) || code >= cthr) return false;
    const uint64_t qh = mix64(d ^ kSlotSalt);
    slot = fastrange32((uint32_t)(qh >> 32), k);
    key = ((uint64_t)code << 32) | (uint32_t)qh;
    return true;
}

// Evaluate up to 64 queued darts, two per lane.
template <bool COUNT, bool RHO0>
__device__ __forceinline__ void drain(int n, Queue &q, const WarpMem &m, int lane, uint32_t k, uint32_t cthr,
                                      unsigned long long &kept) {
    uint32_t s0 = 0, s1 = 0;
    uint64_t k0 = 0, k1 = 0;
    const bool e0 = lane < n && dart_eval<RHO0>(m, q.head + lane, k, cthr, s0, k0);
    const bool e1 = lane + 32 < n && dart_eval<RHO0>(m, q.head + 32 + lane, k, cthr, s1, k1);
    if (e0) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s0]), (unsigned long long)k0);
    if (e1) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s1]), (unsigned long long)k1);
    if (COUNT) kept += (unsigned long long)e0 + (unsigned long long)e1;
    q.head += (uint32_t)n;
    __syncwarp();
}

// Emission state of one lane: the current area's remaining darts.
struct Emit {
    uint64_t c;       // counter of the next dart of the current area
    uint64_t pv;
    uint32_t meta;
    int rem;          // darts of the current area not yet emitted
};

// One emission round: every lane with a pending dart appends it to the queue (slot = rank of
// the lane among emitting lanes), then full batches are evaluated.
template <bool COUNT, bool RHO0>
__device__ __forceinline__ void emit_round(Emit &em, Queue &q, const WarpMem &m, int lane, unsigned lt_mask,
                                           uint32_t k, uint32_t cthr, unsigned long long &kept) {
    const bool has = em.rem > 0;
    const unsigned bal = __ballot_sync(kFull, has);
    if (has) {
        const uint32_t i = (q.tail + __popc(bal & lt_mask)) & (kQueue - 1);
        m.dq_c[i] = em.c;
        m.dq_p[i] = em.pv;
        m.dq_m[i] = (uint16_t)em.meta;
        em.c += kGolden;
        --em.rem;
    }
    q.tail += __popc(bal);
    __syncwarp();
    if (q.tail - q.head >= 64) drain<COUNT, RHO0>(64, q, m, lane, k, cthr, kept);
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
    m.tnu[lane] = n_el ? nutop : -1;
    m.toff[lane] = incl - n_el;
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
// column (w = 0) of rows [rlo(nu), rhi(nu)) with rlo = floor(g_prev 2^nu) (0 on the first
// pass) and rhi = ceil(g 2^nu), so an element's areas form a 1-D sequence.  Tiles whose
// elements all have nu_top <= 31 run it in 32-bit arithmetic: then
// floor(G / 2^(64 - nu)) = hi32(G) >> (32 - nu), the element's area count is
// 1 + nu_top + sum_{nu=1..nu_top} (floor(gm1 / 2^(64-nu)) - floor(gfl_prev / 2^(64-nu))) with
// sum_{nu=1..n} floor(G / 2^(64-nu)) = 2H - popc(H), H = floor(G / 2^(64-n)), and the area
// counter e + gamma (nu 2^58 + r + 1) = e + gamma + gamma r + ((21 nu mod 64) << 58)
// (gamma mod 64 = 21).
struct Walk0S {
    int el, nu, nutop;
    uint32_t r, rhi, vmax, g_hi, glo_hi;
    uint64_t e, F, ctr;

    __device__ static uint32_t rows_hi(uint32_t g_hi, int nu) { return nu ? (g_hi >> (32 - nu)) + 1u : 1u; }
    __device__ static uint32_t rows_lo(uint32_t glo_hi, int nu) { return nu ? (glo_hi >> (32 - nu)) : 0u; }
    __device__ static uint32_t ssum(uint32_t G_hi, int n) {
        if (n <= 0) return 0;
        uint32_t H = G_hi >> (32 - n);
        return 2 * H - (uint32_t)__popc(H);
    }
    __device__ static uint32_t count(int nutop, const PassCut &pc) {
        return 1u + (uint32_t)nutop + ssum((uint32_t)(pc.gm1 >> 32), nutop) - ssum((uint32_t)(pc.gfl_lo >> 32), nutop);
    }
    __device__ void region() {
        r = rows_lo(glo_hi, nu);
        rhi = rows_hi(g_hi, nu);
        vmax = (nu == nutop) ? (uint32_t)(F >> 40) : kUMask;
        ctr = e + kGolden + kGolden * (uint64_t)r + ((uint64_t)((21u * (uint32_t)nu) & 63u) << 58);
    }
    __device__ void load(const WarpMem &m) {
        e = m.te[el];
        F = m.tF[el];
        nutop = m.tnu[el];
    }
    __device__ void locate(uint32_t idx, const WarpMem &m, const PassCut &pc) {
        g_hi = (uint32_t)(pc.gm1 >> 32);
        glo_hi = (uint32_t)(pc.gfl_lo >> 32);
        el = tile_element(m, idx);
        load(m);
        uint32_t li = idx - (uint32_t)m.toff[el];
        for (nu = 0;; ++nu) {
            uint32_t rows = rows_hi(g_hi, nu) - rows_lo(glo_hi, nu);
            if (li < rows) break;
            li -= rows;
        }
        region();
        r += li;
        ctr += kGolden * (uint64_t)li;
    }
    __device__ uint64_t pv() const { return ((uint64_t)r << 24) | vmax; }
    __device__ uint32_t meta() const { return pack_meta(0, nu + 24); }
    __device__ void advance(const WarpMem &m) {
        ++r;
        ctr += kGolden;
        if (r != rhi) return;
        if (++nu > nutop) {
            nu = 0;
            do { ++el; } while (el < 32 && m.tnu[el] < 0);
            if (el >= 32) return;
            load(m);
        }
        region();
    }
};

// ------------------------------------------------------------------------------------------
// Fast-kernel batch emission.  Per tile, every lane walks an equal share of the areas; in each
// iteration every lane hashes one area, and the darts of all 32 areas are written to the
// queue at once (positions from a ballot prefix sum of X < 16), so the warp spends exactly one
// iteration per area slot.  A record is 16 bytes: the dart counter c and
// pvs = r << 24 | vmax | S << 57 (r < 2^31 in the 32-bit walk), rank = (r 2^24 + u) 2^-S.
// ------------------------------------------------------------------------------------------
constexpr int kFastQueue = 128;
constexpr int kRowTab = 40;                       // nu = 0..38 (+1 pad)
constexpr uint64_t kRMask = ((1ull << 55) - 1) & ~(uint64_t)kUMask;

struct FastMem {
    uint64_t *slots, *fq_c, *fq_p, *te;
    uint32_t *tv, *toff, *rlo, *rhi;
    int *tnu;
};

size_t fast_warp_bytes(int k) {
    size_t b = (size_t)k * 8 + 2 * kFastQueue * 8 + 32 * 8 + 3 * 32 * 4 + 2 * kRowTab * 4;
    return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ FastMem carve_fast(unsigned char *base, int k) {
    FastMem m;
    m.slots = reinterpret_cast<uint64_t *>(base);
    m.fq_c = m.slots + k;
    m.fq_p = m.fq_c + kFastQueue;
    m.te = m.fq_p + kFastQueue;
    m.tv = reinterpret_cast<uint32_t *>(m.te + 32);
    m.toff = m.tv + 32;
    m.tnu = reinterpret_cast<int *>(m.toff + 32);
    m.rlo = reinterpret_cast<uint32_t *>(m.tnu + 32);
    m.rhi = m.rlo + kRowTab;
    return m;
}

__device__ __forceinline__ bool fast_eval(const FastMem &m, uint32_t pos, uint32_t k, uint32_t cthr,
                                          uint32_t &slot, uint64_t &key) {
    const uint32_t i = pos & (kFastQueue - 1);
    const uint64_t pvs = m.fq_p[i];
    const uint64_t d = mix64(m.fq_c[i]);
    const uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & kUMask;
    const uint64_t P = (pvs & kRMask) | u;
    const uint32_t code = P ? __float_as_uint(__ull2float_rz(P)) - ((uint32_t)(pvs >> 57) << 23) : 0u;
    if (v > ((uint32_t)pvs & kUMask) || code >= cthr) return false;
    const uint64_t qh = mix64(d ^ kSlotSalt);
    slot = fastrange32((uint32_t)(qh >> 32), k);
    key = ((uint64_t)code << 32) | (uint32_t)qh;
    return true;
}

template <bool COUNT>
__device__ __forceinline__ void fast_drain(int n, Queue &q, const FastMem &m, int lane, uint32_t k, uint32_t cthr,
                                           unsigned long long &kept) {
    uint32_t s0 = 0, s1 = 0;
    uint64_t k0 = 0, k1 = 0;
    const bool e0 = lane < n && fast_eval(m, q.head + lane, k, cthr, s0, k0);
    const bool e1 = lane + 32 < n && fast_eval(m, q.head + 32 + lane, k, cthr, s1, k1);
    if (e0) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s0]), (unsigned long long)k0);
    if (e1) atomicMin(reinterpret_cast<unsigned long long *>(&m.slots[s1]), (unsigned long long)k1);
    if (COUNT) kept += (unsigned long long)e0 + (unsigned long long)e1;
    q.head += (uint32_t)n;
    __syncwarp();
}

// The 1-D walk of a rank-region-0 pass in 32-bit arithmetic (element nu_top <= 31): region nu
// has rows [rlo[nu], rhi[nu]) from the pass table; the area counter is
// e + gamma (nu 2^58 + r + 1) = e + gamma + gamma r + ((21 nu mod 64) << 58) (gamma mod 64 = 21).
struct WalkF {
    int el, nu, nutop;
    uint32_t r, rhi, vtop;
    uint64_t e, ctr, pvr;     // pvr = vmax | S << 57 of the current region

    __device__ void region(const FastMem &m) {
        r = m.rlo[nu];
        rhi = m.rhi[nu];
        pvr = (uint64_t)(nu == nutop ? vtop : kUMask) | ((uint64_t)(nu + 24) << 57);
        ctr = e + kGolden + kGolden * (uint64_t)r + ((uint64_t)((21u * (uint32_t)nu) & 63u) << 58);
    }
    __device__ void load(const FastMem &m) {
        e = m.te[el];
        vtop = m.tv[el];
        nutop = m.tnu[el];
    }
    __device__ void locate(uint32_t idx, const FastMem &m) {
        el = 0;                                   // last element whose offset is <= idx
#pragma unroll
        for (int step = 16; step; step >>= 1) {
            int c = el + step;
            if (c < 32 && m.toff[c] <= idx) el = c;
        }
        load(m);
        uint32_t li = idx - m.toff[el];
        for (nu = 0;; ++nu) {
            uint32_t rows = m.rhi[nu] - m.rlo[nu];
            if (li < rows) break;
            li -= rows;
        }
        region(m);
        r += li;
        ctr += kGolden * (uint64_t)li;
    }
    __device__ uint64_t pvs() const { return pvr | ((uint64_t)r << 24); }
    __device__ void advance(const FastMem &m) {
        ++r;
        ctr += kGolden;
        if (r != rhi) return;
        if (++nu > nutop) {
            nu = 0;
            do { ++el; } while (el < 32 && m.tnu[el] < 0);
            if (el >= 32) return;
            load(m);
        }
        region(m);
    }
};

// One rank-region-0 pass of DartHash over the row in the fast kernel.  Returns 0, an error
// code, or kDefer when a tile is outside the 32-bit walk's range.
template <bool COUNT>
__device__ int fast_pass(const SketchParams &p, int64_t beg, int64_t end, const PassCut &pc, const FastMem &m,
                         int lane, unsigned long long *cnt) {
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t k = (uint32_t)p.k;
    // rows of region nu in this pass: [floor(g_prev 2^nu), ceil(g 2^nu))
    for (int nu = lane; nu < kRowTab; nu += 32) {
        int n = nu > kMaxRegion ? kMaxRegion : nu;
        m.rlo[nu] = n ? (uint32_t)min(pc.gfl_lo >> (64 - n), (uint64_t)0xFFFFFFFFu) : 0u;
        m.rhi[nu] = n ? (uint32_t)min((pc.gm1 >> (64 - n)) + 1, (uint64_t)0xFFFFFFFFu) : 1u;
    }
    const uint32_t g_hi = (uint32_t)(pc.gm1 >> 32), glo_hi = (uint32_t)(pc.gfl_lo >> 32);
    Queue q = {0, 0};
    for (int64_t tile = beg; tile < end; tile += 32) {
        const int64_t pos = tile + lane;
        int nutop = -1;
        uint64_t F = 0, e = 0;
        if (pos < end) {
            nutop = weight_geometry(__float_as_uint(p.weights[pos]), p.t, F);
            if (nutop >= 0) e = mix64(p.sigma + kGolden * ((uint64_t)p.indices[pos] + 1));
        }
        if (__any_sync(kFull, nutop == -2)) return DM_ERANGE;
        if (!__all_sync(kFull, nutop <= 31)) return kDefer;
        // element area count: 1 + nu_top + sum_{nu=1..nu_top} (hi32(gm1) >> (32-nu)) - (hi32(gfl) >> (32-nu)),
        // each sum = 2H - popc(H) with H = hi32(G) >> (32 - nu_top)
        uint64_t n_el = 0;
        if (nutop >= 0) {
            n_el = 1 + (uint64_t)nutop;
            if (nutop > 0) {
                uint32_t H = g_hi >> (32 - nutop), Hl = glo_hi >> (32 - nutop);
                n_el += (2 * (uint64_t)H - __popc(H)) - (2 * (uint64_t)Hl - __popc(Hl));
            }
        }
        uint64_t incl = warp_incl_scan(n_el, lane);
        const uint64_t total = __shfl_sync(kFull, incl, 31);
        if (total >= (1ull << 31)) return kDefer;
        m.te[lane] = e;
        m.tv[lane] = (uint32_t)(F >> 40);
        m.tnu[lane] = n_el ? nutop : -1;
        m.toff[lane] = (uint32_t)(incl - n_el);
        __syncwarp();
        if (total == 0) continue;
        const uint32_t share = (uint32_t)((total + 31) >> 5);
        const uint32_t lo = share * (uint32_t)lane;
        const uint32_t mine = lo < (uint32_t)total ? min(share, (uint32_t)total - lo) : 0u;
        WalkF s;
        if (mine) s.locate(lo, m);
        for (uint32_t it = 0; it < share; ++it) {
            int X = 0;
            uint64_t a = 0, pv = 0;
            if (it < mine) {
                a = mix64(s.ctr);
                X = poisson1((uint32_t)(a >> 32), c_pois);
                pv = s.pvs();
                if (COUNT) { cnt[0]++; cnt[1] += X; }
                if (it + 1 < mine) s.advance(m);
            }
            // prefix sum of X (< 16) over the lanes from four ballots
            const unsigned b0 = __ballot_sync(kFull, X & 1), b1 = __ballot_sync(kFull, X & 2);
            const unsigned b2 = __ballot_sync(kFull, X & 4), b3 = __ballot_sync(kFull, X & 8);
            const uint32_t T = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2) + 8 * __popc(b3);
            if (T == 0) continue;
            const uint32_t ex = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt) + 8 * __popc(b3 & lt);
            // write the darts in queue-sized pieces (one piece unless T is far above its mean)
            for (uint32_t done = 0; done < T;) {
                const uint32_t room = kFastQueue - (q.tail - q.head);
                const uint32_t lim = min(T - done, room);
                uint32_t jlo = done > ex ? done - ex : 0u;
                uint32_t jhi = done + lim > ex ? done + lim - ex : 0u;
                if (jhi > (uint32_t)X) jhi = (uint32_t)X;
                uint64_t c = a + kGolden * (uint64_t)(jlo + 1);
                for (uint32_t j = jlo; j < jhi; ++j, c += kGolden) {
                    const uint32_t i = (q.tail + ex + j - done) & (kFastQueue - 1);
                    m.fq_c[i] = c;
                    m.fq_p[i] = pv;
                }
                q.tail += lim;
                done += lim;
                __syncwarp();
                while (q.tail - q.head >= 64) fast_drain<COUNT>(64, q, m, lane, k, pc.cthr, cnt[2]);
            }
        }
    }
    if (q.tail != q.head) fast_drain<COUNT>((int)(q.tail - q.head), q, m, lane, k, pc.cthr, cnt[2]);
    return 0;
}

// ------------------------------------------------------------------------------------------
// General walk: regions (nu, rho), columns w and rows r.
// ------------------------------------------------------------------------------------------
struct WalkG {
    int el, nu, rho, nutop;
    uint64_t w, r, ncols, rlo, rhi;
    uint64_t e, F, WT, rbase, packhi, ctr;

    __device__ static uint64_t count(int nutop, uint64_t F, const PassCut &pc) {
        uint64_t total = 0;
        for (int n = 0; n <= nutop; ++n)
            for (int h = pc.rho_lo; h <= pc.rho_top; ++h)
                total += cols(n, h, nutop, F) * (rows_hi(pc, n, h) - rows_lo(pc, n, h));
        return total;
    }
    __device__ void region(const PassCut &pc) {
        ncols = cols(nu, rho, nutop, F);
        rlo = rows_lo(pc, nu, rho);
        rhi = rows_hi(pc, nu, rho);
        WT = (nu == nutop) ? (F >> (40 - rho)) : ~0ull;
        rbase = ((1ull << rho) - 1) << (62 - rho);
        packhi = ((uint64_t)nu << 58) | ((uint64_t)rho << 52);
    }
    __device__ void set_ctr() { ctr = e + kGolden * ((packhi | (w << nu) | r) + 1); }
    __device__ void load(const WarpMem &m) {
        e = m.te[el];
        F = m.tF[el];
        nutop = m.tnu[el];
    }
    __device__ void locate(uint64_t idx, const WarpMem &m, const PassCut &pc) {
        el = tile_element(m, idx);
        load(m);
        uint64_t li = idx - m.toff[el];
        for (nu = 0; nu <= nutop; ++nu) {
            bool found = false;
            for (rho = pc.rho_lo; rho <= pc.rho_top; ++rho) {
                region(pc);
                uint64_t nrows = rhi - rlo, c = ncols * nrows;
                if (li < c) {
                    w = li / nrows;
                    r = rlo + (li - w * nrows);
                    found = true;
                    break;
                }
                li -= c;
            }
            if (found) break;
        }
        set_ctr();
    }
    __device__ uint64_t pv() const {
        return rbase + (r << (62 - nu)) + min(WT - (w << 24), (uint64_t)kUMask);
    }
    __device__ uint32_t meta() const { return pack_meta(38 - nu, 62 - rho); }
    __device__ void advance(const WarpMem &m, const PassCut &pc) {
        ++r;
        ctr += kGolden;
        if (r < rhi) return;
        ++w;
        if (w >= ncols) {
            w = 0;
            if (++rho > pc.rho_top) {
                rho = pc.rho_lo;
                if (++nu > nutop) {
                    nu = 0;
                    do { ++el; } while (el < 32 && m.tnu[el] < 0);
                    if (el >= 32) return;         // past the tile: the lane is done
                    load(m);
                }
            }
            region(pc);
        }
        r = rlo;
        set_ctr();
    }
};

// Emission loop over one tile with walk W (W::locate positions the walk at a lane's first
// area, W::advance moves to the next): each lane hashes its next area once the darts of the
// previous one are emitted, and emits at most one dart per round.
template <class W, class Idx, bool COUNT, bool RHO0, class Adv>
__device__ __forceinline__ void run_tile(W &s, Idx left, Adv advance, Queue &q, const WarpMem &m, int lane,
                                         unsigned lt_mask, uint32_t k, uint32_t cthr, unsigned long long *cnt) {
    Emit em;
    em.rem = 0;
    while (__any_sync(kFull, left > 0 || em.rem > 0)) {
        if (em.rem == 0 && left > 0) {
            const uint64_t a = mix64(s.ctr);
            em.rem = poisson1((uint32_t)(a >> 32), c_pois);
            em.c = a + kGolden;
            em.pv = s.pv();
            em.meta = s.meta();
            if (COUNT) { cnt[0]++; cnt[1] += em.rem; }
            if (--left) advance(s);
        }
        emit_round<COUNT, RHO0>(em, q, m, lane, lt_mask, k, cthr, cnt[2]);
    }
}

// One pass of DartHash over the row; RHO0 passes have a rank limit below 1.  Returns 0 or an
// error code.
template <bool RHO0, bool COUNT>
__device__ int darthash_pass(const SketchParams &p, int64_t beg, int64_t end, const PassCut &pc,
                             const WarpMem &m, int lane, unsigned long long *cnt) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t k = (uint32_t)p.k;
    Queue q = {0, 0};
    for (int64_t tile = beg; tile < end; tile += 32) {
        int nutop;
        uint64_t F, e;
        const bool ok = element_setup(p, tile + lane, end, nutop, F, e);
        if (__any_sync(kFull, !ok)) return DM_ERANGE;
        if (RHO0) {
            // 32-bit walk; a tile outside its range sends the whole set to the general kernel
            if (!__all_sync(kFull, nutop <= 31)) return kDefer;
            const uint64_t total = publish_tile(m, lane, nutop, F, e, nutop >= 0 ? Walk0S::count(nutop, pc) : 0);
            if (total == 0) continue;
            if (total >= (1ull << 31)) return kDefer;
            const uint32_t share = (uint32_t)((total + 31) >> 5);
            const uint32_t lo = share * (uint32_t)lane;
            uint32_t left = lo < (uint32_t)total ? min(share, (uint32_t)total - lo) : 0u;
            Walk0S s;
            if (left) s.locate(lo, m, pc);
            run_tile<Walk0S, uint32_t, COUNT, RHO0>(s, left, [&](Walk0S &w) { w.advance(m); }, q, m, lane,
                                                     lt_mask, k, pc.cthr, cnt);
        } else {
            const uint64_t total = publish_tile(m, lane, nutop, F, e, nutop >= 0 ? WalkG::count(nutop, F, pc) : 0);
            if (total == 0) continue;
            const uint64_t share = (total + 31) >> 5;
            const uint64_t lo = share * lane;
            uint64_t left = lo < total ? min(share, total - lo) : 0;
            WalkG s;
            if (left) s.locate(lo, m, pc);
            run_tile<WalkG, uint64_t, COUNT, RHO0>(s, left, [&](WalkG &w) { w.advance(m, pc); }, q, m, lane,
                                                    lt_mask, k, pc.cthr, cnt);
        }
    }
    if (q.tail != q.head) drain<COUNT, RHO0>((int)(q.tail - q.head), q, m, lane, k, pc.cthr, cnt[2]);
    return 0;
}

// MODE 0 (fast): every pass whose rank limit is below 1 runs the 1-D walk; a set needing a
// limit >= 1 is appended to the general queue and left to MODE 1.
// MODE 1 (general): sets are taken from the queue and computed from the first pass with the
// general walk.  Both give the same bits for a set (the output does not depend on the limits).
// Warps are persistent and claim work items from a global counter.
template <bool BBIT, bool COUNT, int MODE>
__global__ void __launch_bounds__(256, MODE == 0 ? 4 : 2) sketch_kernel(const SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wbytes = MODE == 0 ? p.warp_bytes_fast : p.warp_bytes;
    WarpMem m = carve(smem + (size_t)wib * wbytes, p.k);
    FastMem fm = carve_fast(smem + (size_t)wib * wbytes, p.k);
    const uint32_t k = (uint32_t)p.k;
    const int64_t n_work = MODE == 0 ? p.n_sets : (int64_t)*p.queue_count;
    unsigned int *next = p.work_next + MODE;
    for (;;) {
        unsigned int wi = 0;
        if (lane == 0) wi = atomicAdd(next, 1u);
        wi = __shfl_sync(kFull, wi, 0);
        if ((int64_t)wi >= n_work) break;
        const int64_t set = MODE == 0 ? (int64_t)wi : (int64_t)p.queue[wi];
        const int64_t beg = p.indptr[set], end = p.indptr[set + 1];
        // ||x||_1 and input validation
        float l1 = 0.f;
        bool bad = false;
        for (int64_t i = beg + lane; i < end; i += 32) {
            float x = p.weights[i];
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
                // the fast kernel only runs rank-region-0 passes; the general kernel runs the
                // general walk on every pass (it is correct for any limit)
                err = MODE == 0 ? fast_pass<COUNT>(p, beg, end, pc, fm, lane, cnt)
                                : darthash_pass<false, COUNT>(p, beg, end, pc, m, lane, cnt);
                ++passes;
                if (err == kDefer) { err = 0; deferred = true; break; }
                if (err) break;
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
    size_t smem = (size_t)(MODE == 0 ? p.warp_bytes_fast : p.warp_bytes) * p.warps_per_block;
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
    // queue count and the two work counters are contiguous
    cudaError_t e = cudaMemsetAsync(p.queue_count, 0, 4 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if ((e = launch_mode<0>(p, bbit, count, grid_fast, st)) != cudaSuccess) return e;
    return launch_mode<1>(p, bbit, count, grid_general, st);
}

}  // namespace dm

namespace dm {
int sketch_blocks_per_sm(int mode, bool bbit, int warps_per_block, size_t smem) {
    int nb = 0;
    const void *fn;
    if (mode == 0) fn = bbit ? (const void *)sketch_kernel<true, false, 0> : (const void *)sketch_kernel<false, false, 0>;
    else fn = bbit ? (const void *)sketch_kernel<true, false, 1> : (const void *)sketch_kernel<false, false, 1>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * warps_per_block, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}
}  // namespace dm
