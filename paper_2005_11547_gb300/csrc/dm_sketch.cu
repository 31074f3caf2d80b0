// DartMinHash kernels for sm_103a: one warp per weighted set.
//
// Per set (Christiani, arXiv 2005.11547, Theorem 1): compute ||x||_1, set the rank limit
// theta = phi0 / ||x||_1, run DartHash (Algorithm 1) for darts of rank < theta and hand every
// kept dart to a sink; while the sink is not filled, double theta and enumerate only the areas
// that reach above the previous limit (the band).
//   * SketchSink: the dart is hashed to one of k buckets, the bucket keeps the minimum key
//     (Theorem 1's k independent minhashes; b-bit packing in the epilogue, Section 1.1).
//   * LshSink: the dart is hashed to one of L buckets, the bucket keeps its K smallest keys,
//     and table l's value is a hash of them in increasing order ((L, K) LSH, Section 3).
//
// GPU mapping
//  * Persistent warps claim sets from a global counter, so a set that needs a second pass
//    never holds idle warps of its block.
//  * Two kernels per call.  The fast kernel runs passes whose limit is below 1 (rank region 0
//    only: each element's areas are a 1-D sequence of rows) in 32-bit arithmetic; a set that
//    needs anything else is appended to a device queue that the general kernel (all regions,
//    64-bit) then computes from its first pass.  The output does not depend on the limits, so
//    both give the same bits.
//  * Elements are taken 32 at a time (a tile, one lane each).  Each lane computes its
//    element's area count for the pass in closed form; a warp scan flattens the tile's areas
//    and every lane walks a contiguous, equal share of them.
//  * Each area costs one hash (its Poisson count X), each dart one (its U, V), each kept dart
//    one (its bucket and fingerprint).  In the fast path every step of the warp runs one kind
//    of hash on all lanes: area steps (with the first dart of each area), dart steps over a
//    per-warp queue of areas with more darts, and bucket steps over a queue of kept darts, so
//    the variable Poisson counts and keep decisions do not leave lanes idle.
#include <mutex>

#include "dm_device.cuh"
#include "dm_internal.h"

namespace dm {

__constant__ uint32_t c_pois[12];

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMaxPasses = 21;     // phi0 * 2^20 at most (Theorem 1's loop limit)
constexpr int kDefer = -1;         // a pass the fast kernel leaves to the general kernel
// batched form: hist[0..96) bin counts, [96..192) bin cursors, [192..195) class totals
constexpr int kClasses = 3, kBins = 32, kCursors = kClasses * kBins, kTotals = 2 * kClasses * kBins;
constexpr int kDeferNext = kTotals + kClasses;   // hist word: next deferred set of the general kernel
constexpr size_t kHeaderBytes = 1024;   // queue count, 3 work counters, histogram, totals
static_assert((4 + kDeferNext + 1) * sizeof(unsigned int) <= kHeaderBytes, "header holds every counter");
constexpr int kMaxDevices = 64;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// ==========================================================================================
// Sinks
// ==========================================================================================

// LSH: L buckets of K sorted keys, then the L counts.
size_t lsh_sink_bytes(int L, int K) { return ((size_t)L * K * 8 + (size_t)L * 4 + 15) & ~(size_t)15; }

// k buckets, each the minimum key of the darts hashed to it (Theorem 1).  Two layouts, with the
// same bits:
//  * shared: the k 64-bit minima live in shared memory (8 k bytes per warp);
//  * key row (p.key_row, the default when keys go to device memory): shared memory holds a
//    16-bit filter per bucket (2 k bytes) and the 64-bit minimum goes straight to the set's
//    output row in global memory (L2-resident while the set runs).  The filter is the high half
//    of the rank code of a dart already in the row's minimum (see put), so a candidate whose
//    high half exceeds it cannot be the minimum; the others reach the row, whose 64-bit atomic
//    minimum decides.
// 0xFFFF marks an empty bucket's filter: a kept dart's code is below bits(theta) < 0x7F800000.
__host__ __device__ size_t sketch_sink_bytes(int k, bool key_row) {
    return ((size_t)k * (key_row ? 2 : 8) + 15) & ~(size_t)15;
}

template <bool KEYROW>
struct SketchSinkT {
    uint64_t *slots;                              // shared layout: the k minima
    uint16_t *codes;                              // key-row layout: a filter per bucket (see put)
    uint64_t *row;                                // key-row layout: the set's output row
    uint32_t k;
    uint32_t sbase;                               // shared-space address of the bucket array
    static constexpr bool kLowerCut = false;      // min is idempotent: band overlap is harmless

    __device__ void bind(unsigned char *base, const SketchParams &p) {
        slots = reinterpret_cast<uint64_t *>(base);
        codes = reinterpret_cast<uint16_t *>(base);
        k = (uint32_t)p.k;
        sbase = (uint32_t)__cvta_generic_to_shared(base);
        row = nullptr;
    }
    __device__ void set_row(const SketchParams &p, int64_t set) {
        if constexpr (KEYROW) row = p.out_keys + set * (int64_t)k;
    }
    __device__ void reset(int lane) {
        if constexpr (KEYROW)
            for (uint32_t j = lane; j < k; j += 32) {
                codes[j] = (uint16_t)0xFFFFu;
                row[j] = ~0ull;
            }
        else
            for (uint32_t j = lane; j < k; j += 32) slots[j] = ~0ull;
        __syncwarp();
    }
    __device__ __forceinline__ bool put(uint64_t qh, uint32_t code) {
        const uint32_t slot = fastrange32((uint32_t)(qh >> 32), k);
        const uint64_t key = ((uint64_t)code << 32) | (uint32_t)qh;
        if (!DM_EXPECT(slot < k)) return false;
        if constexpr (KEYROW) {
            // The filter holds the high 16 bits of the code of a dart already in the bucket's
            // row minimum, so it is at least the high half of the row minimum's code; a dart
            // whose high half exceeds it cannot lower the minimum and is dropped.  Lanes may race
            // on the plain store: whichever value is left is such a code, so the filter only ever
            // lets more darts through to the exact 64-bit atomic minimum on the row.
            const uint32_t c16 = code >> 16, cur = codes[slot];
            if (c16 <= cur) {
                if (c16 < cur) codes[slot] = (uint16_t)c16;
                atomicMin(reinterpret_cast<unsigned long long *>(&row[slot]), (unsigned long long)key);
            }
        } else {
            shared_min_u64(sbase + 8u * slot, key);
        }
        return false;
    }
    // called by the whole warp; lanes with have = true hold a kept dart
    __device__ __forceinline__ void put_batch(bool have, uint64_t qh, uint32_t code, int) {
        if (have) put(qh, code);
    }
    __device__ bool empty_bucket(uint32_t j) const {
        if constexpr (KEYROW) return codes[j] == (uint16_t)0xFFFFu;        // codes are below 0x7F80_0000
        return slots[j] == ~0ull;
    }
    __device__ bool filled(int lane) {
        bool empty = false;
        for (uint32_t j = lane; j < k; j += 32) empty |= empty_bucket(j);
        return !__any_sync(kFull, empty);
    }
    __device__ void clear_to_error(int lane) {
        for (uint32_t j = lane; j < k; j += 32) {
            if constexpr (KEYROW) row[j] = ~0ull;
            else slots[j] = ~0ull;
        }
        __syncwarp();
    }
    // the final key of bucket j (the row is read from L2: the global minima were updated there)
    __device__ __forceinline__ uint64_t key(uint32_t j) const {
        if constexpr (KEYROW) return __ldcg(reinterpret_cast<const unsigned long long *>(&row[j]));
        return slots[j];
    }
    template <bool BBIT>
    __device__ void finish(const SketchParams &p, int64_t set, bool err, int lane) {
        if (!KEYROW && p.out_keys)
            for (uint32_t j = lane; j < k; j += 32) p.out_keys[set * (int64_t)k + j] = slots[j];
        if (!BBIT) return;
        const int b = p.b;
        const uint64_t bmask = (1ull << b) - 1;
        uint64_t *ow = p.out_words + set * (int64_t)p.words;
        if (err) {
            for (int wd = lane; wd < p.words; wd += 32) ow[wd] = ~0ull;   // error rows are all ones
        } else if (b == 1) {
            for (uint32_t j0 = 0; j0 < k; j0 += 64) {
                uint32_t j1 = j0 + lane, j2 = j0 + 32 + lane;
                bool b1 = j1 < k && (mix64(key(j1) ^ kBbitSalt) & 1);
                bool b2 = j2 < k && (mix64(key(j2) ^ kBbitSalt) & 1);
                unsigned lo = __ballot_sync(kFull, b1), hi = __ballot_sync(kFull, b2);
                if (lane == 0) ow[j0 >> 6] = (uint64_t)lo | ((uint64_t)hi << 32);
            }
        } else {
            const int g = 64 / b;                    // slots per word, 2..32
            for (uint32_t j0 = 0; j0 < k; j0 += 32) {
                uint32_t j = j0 + lane;
                uint64_t v = 0;
                if (j < k) v = (mix64(key(j) ^ kBbitSalt) & bmask) << ((j * (uint32_t)b) & 63);
                for (int o = 1; o < g; o <<= 1) v |= __shfl_xor_sync(kFull, v, o);
                if ((lane & (g - 1)) == 0 && j < k) ow[(j * (uint32_t)b) >> 6] = v;
            }
        }
    }
};
using SketchSink = SketchSinkT<false>;   // bucket minima in shared memory
using RowSink = SketchSinkT<true>;       // 16-bit filters in shared memory, minima in the output row

// L buckets, each the K smallest keys of the darts hashed to it ((L, K) LSH), kept sorted in
// shared memory.  A batch of kept darts is inserted by the whole warp: darts of different buckets
// go in at once, and darts of one bucket (grouped by __match_any_sync) take turns, so no bucket is
// written by two lanes at a time.  A key at or above a full bucket's K-th key is dropped.  Band
// passes must not add a dart twice, so darts below the previous limit are cut before they reach
// the sink.  Table l's value is a hash of bucket l's K keys in increasing order.
struct LshSink {
    uint64_t *buf;                                // [L][K], ascending
    uint32_t *cnt;                                // [L]
    uint32_t L, K;
    static constexpr bool kLowerCut = true;

    __device__ void bind(unsigned char *base, const SketchParams &p) {
        L = (uint32_t)p.k;
        K = (uint32_t)p.K;
        buf = reinterpret_cast<uint64_t *>(base);
        cnt = reinterpret_cast<uint32_t *>(buf + (size_t)L * K);
    }
    __device__ void set_row(const SketchParams &, int64_t) {}
    __device__ void reset(int lane) {
        for (uint32_t b = lane; b < L; b += 32) cnt[b] = 0;
        __syncwarp();
    }
    // insertion of key into bucket b's sorted keys (the caller owns bucket b for this call)
    __device__ __forceinline__ void insert(uint32_t b, uint64_t key) {
        if (!DM_EXPECT(b < L && cnt[b] <= K)) return;
        uint64_t *v = buf + (size_t)b * K;
        uint32_t n = cnt[b];
        if (n == K) {
            if (key >= v[K - 1]) return;
            n = K - 1;                            // the largest key leaves
        } else {
            cnt[b] = n + 1;
        }
        uint32_t j = n;
        while (j > 0 && v[j - 1] > key) {
            v[j] = v[j - 1];
            --j;
        }
        v[j] = key;
    }
    // Called by the whole warp; lanes with have = true hold a kept dart (bucket hash qh, code).
    __device__ __forceinline__ void put_batch(bool have, uint64_t qh, uint32_t code, int lane) {
        const uint32_t b = fastrange32((uint32_t)(qh >> 32), L);
        const uint64_t key = ((uint64_t)code << 32) | (uint32_t)qh;
        // a stale look at the K-th key only lets more darts through; insert decides exactly
        const bool go = have && (cnt[b] < K || key < buf[(size_t)b * K + K - 1]);
        const unsigned grp = __match_any_sync(kFull, go ? b : L + (uint32_t)lane);
        const uint32_t rank = __popc(grp & ((1u << lane) - 1u));
        const uint32_t rounds = __reduce_max_sync(kFull, go ? (uint32_t)__popc(grp) : 0u);
        for (uint32_t it = 0; it < rounds; ++it) {
            if (go && rank == it) insert(b, key);
            __syncwarp();
        }
    }
    __device__ bool filled(int lane) {
        bool lack = false;
        for (uint32_t b = lane; b < L; b += 32) lack |= cnt[b] < K;
        return !__any_sync(kFull, lack);
    }
    __device__ void clear_to_error(int) {}
    template <bool BBIT>
    __device__ void finish(const SketchParams &p, int64_t set, bool err, int lane) {
        uint32_t *o = p.out_lsh + set * (int64_t)L;
        for (uint32_t b = lane; b < L; b += 32) {
            if (err || cnt[b] < K) {                     // error, or a set with no positive weight
                o[b] = 0xFFFFFFFFu;
                continue;
            }
            const uint64_t *v = buf + (size_t)b * K;
            uint64_t h = kLshInit;
            for (uint32_t m = 0; m < K; ++m) h = mix64(h ^ v[m]);
            o[b] = (uint32_t)(h >> 32);
        }
    }
};

// The k smallest keys of a set's darts (Section 3, "Bottom-k minhash": t = k, phi raised until
// at least k darts).  Candidates (keys below tau) are appended to a buffer of C slots; when a
// batch of at most 32 puts brings it within 32 of full, the warp sorts it (bitonic) and keeps
// the k smallest, tau becoming the k-th.  Band passes must not add a dart twice, so darts
// below the previous limit are cut.
__host__ __device__ inline uint32_t bottomk_cap(int k) {
    uint32_t c = 64;
    while (c < 2u * (uint32_t)k || c < (uint32_t)k + 32u) c <<= 1;
    return c;
}
size_t bottomk_sink_bytes(int k) { return (size_t)bottomk_cap(k) * 8 + 16; }

struct BottomKSink {
    uint64_t *buf, *tau;
    uint32_t *cnt;
    uint32_t k, C;
    static constexpr bool kLowerCut = true;

    __device__ void bind(unsigned char *base, const SketchParams &p) {
        k = (uint32_t)p.k;
        C = bottomk_cap(p.k);
        buf = reinterpret_cast<uint64_t *>(base);
        tau = buf + C;
        cnt = reinterpret_cast<uint32_t *>(tau + 1);
    }
    __device__ void set_row(const SketchParams &, int64_t) {}
    __device__ void reset(int lane) {
        if (lane == 0) {
            *cnt = 0;
            *tau = ~0ull;
        }
        __syncwarp();
    }
    // Returns true when the buffer is within 32 of full: the batch ends with a compaction.
    __device__ __forceinline__ bool put(uint64_t qh, uint32_t code) {
        const uint64_t key = ((uint64_t)code << 32) | (uint32_t)qh;
        if (key >= *tau) return false;
        const uint32_t pos = atomicAdd(cnt, 1u);          // < C: at most 32 puts per batch
        if (DM_EXPECT(pos < C)) buf[pos] = key;
        return pos + 33 > C;
    }
    __device__ void compact(int lane) {
        __syncwarp();
        const uint32_t n = *cnt;
        for (uint32_t j = n + (uint32_t)lane; j < C; j += 32) buf[j] = ~0ull;
        __syncwarp();
        warp_bitonic_sort(buf, C, lane);
        if (lane == 0) {
            *cnt = n < k ? n : k;
            if (n >= k) *tau = buf[k - 1];
        }
        __syncwarp();
    }
    // called by the whole warp with at most 32 darts; lanes with have = true hold one
    __device__ __forceinline__ void put_batch(bool have, uint64_t qh, uint32_t code, int lane) {
        const bool need = have && put(qh, code);
        __syncwarp();
        if (__any_sync(kFull, need)) compact(lane);
    }
    __device__ bool filled(int) { return *cnt >= k; }
    __device__ void clear_to_error(int) {}
    template <bool BBIT>
    __device__ void finish(const SketchParams &p, int64_t set, bool err, int lane) {
        compact(lane);
        const uint32_t n = *cnt;
        uint64_t *o = p.out_keys + set * (int64_t)k;
        for (uint32_t j = (uint32_t)lane; j < k; j += 32) o[j] = (!err && j < n) ? buf[j] : ~0ull;
    }
};

// ==========================================================================================
// Fast path: passes with a rank limit theta <= 1.  Every region (nu, 0) is one column of rows
// [rlo(nu), rhi(nu)) with rlo = floor(g_prev 2^nu) (0 on the first pass) and rhi =
// ceil(g 2^nu), so an element's areas form a 1-D sequence.  For elements with nu_top <= 31,
// floor(G / 2^(64 - nu)) = hi32(G) >> (32 - nu), and the element's area count is
// 1 + nu_top + sum_{nu=1..nu_top} (floor(gm1 / 2^(64-nu)) - floor(gfl_prev / 2^(64-nu))) with
// sum_{nu=1..n} floor(G / 2^(64-nu)) = 2H - popc(H), H = floor(G / 2^(64-n)).  The area counter
// e + gamma (nu 2^58 + r + 1) is e + kt[nu] + gamma (r - rlo[nu]) with the per-pass table
// kt[nu] = gamma (1 + rlo[nu]) + ((21 nu mod 64) << 58) (gamma mod 64 = 21).  Tiles with an
// element beyond nu_top = 31 send the set to the general kernel.
//
// Step loop.  The areas of a segment (kSegTiles tiles of 32 elements) are split into 32 equal
// contiguous shares, one per lane, and the warp runs steps of three kinds.  Each kind is chosen
// for the whole warp, so every lane with work runs the same hash at the same time:
//  * area step (every lane on its next area): the area hash a gives the Poisson count X, and
//    the first dart's hash M(a + gamma) is evaluated at once (weight and rank tests).  A kept
//    dart goes to the kept queue; an area with X >= 2 goes to the dart queue with the counter
//    of its second dart (j = 1) and the area's Poisson uniform.
//  * dart step (32 queued areas): dart j of each is hashed and tested; the area goes back to
//    the dart queue when dart j + 1 exists (X > j + 1: the uniform reaches T[j + 1]).
//  * bucket step (32 queued kept darts): the bucket/fingerprint hash, the rank code and the
//    sink.
// A queue is served as soon as it holds 32 entries, so neither exceeds 64; both carry over
// from one segment to the next and are drained at the end of the pass.  Only the last steps
// of a pass (the drain) and the shorter share of a segment's last lanes run on part of the warp.
//
// Rank test in integers: a dart of row r has rank (r 2^24 + u) 2^-S, S = nu + 24, and its code
// (binary32, rounded toward zero) is below bits(theta) iff r 2^24 + u < ceil(theta 2^S) =
// pthr[nu] (theta is a binary32 value, so rounding toward zero cannot cross it).  Every row of a
// region but the last passes whatever u is (pthr > (rhi - 1) 2^24); the last row passes iff
// u < lastthr[nu] = pthr[nu] - (rhi - 1) 2^24, which lies in (0, 2^24].  Likewise the previous
// pass's limit cuts only the first row rlo, at u >= firstlo[nu] = ceil(theta_prev 2^S) - rlo 2^24,
// for the sinks that must not see a dart twice.
// ==========================================================================================
constexpr int kSegTiles = 2, kSeg = 32 * kSegTiles;
constexpr int kFastRegions = 32;      // weight regions nu = 0..31 of the fast path
static_assert(kFastRegions == 32, "one region per lane; WalkF::locate searches 32 regions");
constexpr int kQ = 64;                // capacity of each step queue (served at 32)

// Per-pass record of weight region nu: the area counter offset kt, the u limit of its last row
// and the u floor of its first row (RegA); its first row and row end, and per segment the number
// of its elements and the offset of its first area in the segment (RegB).
struct RegA {
    uint64_t kt;
    uint32_t lastthr, firstlo;
};
struct RegB {
    uint32_t rlo, rhi, cnt, C;
};
// Per-element record of a segment (16 bytes, one load): element key and vtop | nu_top << 24.
struct ElRec {
    uint64_t e;
    uint32_t pad, vn;
};

struct FastMem {
    RegA *ra;                           // [kFastRegions]
    ElRec *el;                          // [kSeg]
    uint4 *kq;                          // kept queue [kQ]: dart hash (low, high word), row r, region nu
    uint4 *xp;                          // dart queue [kQ]: uthr | j << 26, vmax | nu << 24, r, Poisson uniform
    uint64_t *xo;                       // dart queue [kQ]: counter of the area's dart j
    uint32_t *xl;                       // dart queue [kQ]: u floor of the area (sinks with a lower cut)
    RegB *rb;                           // [kFastRegions]
};

constexpr size_t kFastPathBytes = (size_t)kFastRegions * (sizeof(RegA) + sizeof(RegB)) +
                                  (size_t)kSeg * sizeof(ElRec) + (size_t)kQ * (16 + 16 + 8 + 4);
static_assert(sizeof(RegA) == 16 && sizeof(RegB) == 16 && sizeof(ElRec) == 16, "record layout");
static_assert(kFastPathBytes % 16 == 0, "fast-path tables keep 16-byte alignment");

__device__ __forceinline__ FastMem carve_fast(unsigned char *base) {
    FastMem m;
    m.ra = reinterpret_cast<RegA *>(base);
    m.el = reinterpret_cast<ElRec *>(m.ra + kFastRegions);
    m.kq = reinterpret_cast<uint4 *>(m.el + kSeg);
    m.xp = m.kq + kQ;
    m.xo = reinterpret_cast<uint64_t *>(m.xp + kQ);
    m.xl = reinterpret_cast<uint32_t *>(m.xo + kQ);
    m.rb = reinterpret_cast<RegB *>(m.xl + kQ);
    return m;
}

// ceil(value(bits) 2^S) for a positive finite binary32 below 2 and 24 <= S <= 63 (< 2^40 here).
__device__ __forceinline__ uint64_t ceil_scaled(uint32_t bits, int S) {
    if (bits == 0) return 0;
    const uint32_t ex = bits >> 23, fr = bits & 0x7FFFFFu;
    const uint64_t m = ex ? (uint64_t)(fr | 0x800000u) : (uint64_t)fr;
    const int sh = (ex ? (int)ex - 150 : -149) + S;
    if (sh >= 0) return m << sh;
    if (sh <= -24) return 1;                      // 0 < m 2^sh < 1
    return (m + (1ull << -sh) - 1) >> -sh;
}

// The walk over a segment's areas in region-major order: weight region nu, then the region's
// elements (sorted by nu_top, descending, so region nu's elements are the first cnt(nu)), then
// rows.  Every element of a region has the same rows, so a one-row region costs one element
// step per area, and a lane's share rarely crosses a region.
struct WalkF {
    int nu, q, qend;
    uint32_t r, rlo, rhi, vmax, lastthr, firstlo;
    uint64_t kt, ctr;

    __device__ __forceinline__ void region(const FastMem &m) {
        if (!DM_EXPECT(nu >= 0 && nu < kFastRegions)) nu = 0;
        const uint4 a = *reinterpret_cast<const uint4 *>(&m.ra[nu]);          // kt, lastthr, firstlo
        const uint4 b = *reinterpret_cast<const uint4 *>(&m.rb[nu]);          // rlo, rhi, cnt, C
        kt = ((uint64_t)a.y << 32) | a.x;
        lastthr = a.z;
        firstlo = a.w;
        rlo = b.x;
        rhi = b.y;
        qend = (int)b.z;
    }
    // element q of region nu at row r: counter e + kt + gamma (r - rlo); the v limit of the
    // element's last region
    __device__ __forceinline__ void element(const FastMem &m) {
        if (!DM_EXPECT(q >= 0 && q < kSeg)) q = 0;
        const uint4 e = *reinterpret_cast<const uint4 *>(&m.el[q]);
        ctr = (((uint64_t)e.y << 32) | e.x) + kt + kGolden * (uint64_t)(r - rlo);
        vmax = (int)(signed char)(e.w >> 24) == nu ? (e.w & kUMask) : kUMask;
    }
    // position the walk on area idx of the segment (idx < its total)
    __device__ void locate(uint32_t idx, const FastMem &m) {
        nu = 0;                                   // last region whose first area is <= idx
        for (int step = kFastRegions / 2; step; step >>= 1)
            if (m.rb[nu + step].C <= idx) nu += step;
        region(m);
        const uint32_t off = idx - m.rb[nu].C, rows = rhi - rlo;
        q = (int)(off / rows);
        r = rlo + (off - (uint32_t)q * rows);
        element(m);
    }
    // Next area.  Every region of a pass has at least one row (rlo = floor(g_prev 2^nu) <
    // ceil(g 2^nu) = rhi because g_prev < g).
    __device__ __forceinline__ void advance(const FastMem &m) {
        ++r;
        ctr += kGolden;
        if (r == rhi) {
            if (++q == qend) {
                ++nu;
                q = 0;
                region(m);
            }
            r = rlo;
            element(m);
        }
    }
};

// One rank-region-0 pass over tiles first, first + stride, ... of the row [.., end).  The areas
// of each segment are split among nparts warps (this one is number part), 32 lanes each.
// Returns 0, an error code, or kDefer.
template <class Sink, bool COUNT>
__device__ int fast_pass(const SketchParams &p, int64_t first, int64_t stride, int64_t end, const PassCut &pc,
                         const FastMem &m, Sink &sink, int lane, unsigned long long *cnt, int escale = 0,
                         int part = 0, int nparts = 1) {
    constexpr bool LOWER = Sink::kLowerCut;
    __syncwarp();
    uint32_t myrows;                             // rows of region nu = lane in this pass
    {   // per-pass region table, one region per lane
        const int nu = lane;
        const uint32_t lo = nu ? (uint32_t)(pc.gfl_lo >> (64 - nu)) : 0u;
        const uint32_t hi = nu ? (uint32_t)((pc.gm1 >> (64 - nu)) + 1) : 1u;
        const uint64_t pthr = ceil_scaled(pc.cthr, nu + 24), plo = ceil_scaled(pc.cthr_lo, nu + 24);
        m.ra[nu].kt = kGolden * (1ull + lo) + ((uint64_t)((21u * (uint32_t)nu) & 63u) << 58);
        m.ra[nu].lastthr = (uint32_t)(pthr - ((uint64_t)(hi - 1) << 24));
        m.ra[nu].firstlo = (uint32_t)(plo - ((uint64_t)lo << 24));
        m.rb[nu].rlo = lo;
        m.rb[nu].rhi = hi;
        myrows = hi - lo;
    }
    const unsigned lt = (1u << lane) - 1u;
    uint32_t kh = 0, kt = 0, xh = 0, xt = 0;     // kept and dart queues: heads and tails

    auto push_kept = [&](bool keep, uint64_t d, uint32_t r, uint32_t nu) {
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) m.kq[(kt + __popc(km & lt)) & (kQ - 1)] = make_uint4((uint32_t)d, (uint32_t)(d >> 32), r, nu);
        kt += __popc(km);
        (void)DM_EXPECT(kt - kh <= (uint32_t)kQ);     // the ring never overwrites an unserved entry
        if (COUNT && keep) cnt[2]++;
    };
    auto push_darts = [&](bool more, uint64_t op, uint32_t w0, uint32_t w1, uint32_t r, uint32_t up, uint32_t ulo) {
        const unsigned xm = __ballot_sync(kFull, more);
        if (more) {
            const uint32_t i = (xt + __popc(xm & lt)) & (kQ - 1);
            m.xo[i] = op;
            m.xp[i] = make_uint4(w0, w1, r, up);
            if constexpr (LOWER) m.xl[i] = ulo;
        }
        xt += __popc(xm);
        (void)DM_EXPECT(xt - xh <= (uint32_t)kQ);
    };
    // bucket step over the n (<= 32) oldest kept darts
    auto kept_step = [&](uint32_t n) {
        __syncwarp();
        const bool v = (uint32_t)lane < n;
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (v) q = m.kq[(kh + (uint32_t)lane) & (kQ - 1)];
        kh += n;
        const uint64_t d = ((uint64_t)q.y << 32) | q.x;
        const uint64_t h = mix64(d ^ kSlotSalt);
        // binary32 code of rank = P 2^-S rounded toward zero: exact u64 -> f32 conversion in
        // round-toward-zero mode, then the exponent lowered by S
        const uint64_t P = ((uint64_t)q.z << 24) | (uint32_t)(d >> 40);
        const uint32_t code = P ? __float_as_uint(__ull2float_rz(P)) - ((q.w + 24u) << 23) : 0u;
        sink.put_batch(v, h, code, lane);
        __syncwarp();
    };
    // dart step over the n (<= 32) oldest queued areas
    auto dart_step = [&](uint32_t n) {
        __syncwarp();
        const bool v = (uint32_t)lane < n;
        uint64_t op = 0;
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        uint32_t lo = 0;
        if (v) {
            const uint32_t i = (xh + (uint32_t)lane) & (kQ - 1);
            op = m.xo[i];
            x = m.xp[i];
            if constexpr (LOWER) lo = m.xl[i];
        }
        xh += n;
        __syncwarp();                             // every lane has read its entry before any push
        const uint64_t d = mix64(op);
        const uint32_t u = (uint32_t)(d >> 40), vv = (uint32_t)(d >> 16) & kUMask;
        bool keep = v && u < (x.x & 0x3FFFFFFu) && vv <= (x.y & kUMask);
        if constexpr (LOWER) keep = keep && u >= lo;
        push_kept(keep, d, x.z, x.y >> 24);
        // dart j + 1 exists iff X > j + 1, i.e. the area's Poisson uniform reaches T[j + 1]
        const uint32_t jn = (x.x >> 26) + 1u;
        const bool more = v && jn < 12u && x.w >= c_pois[jn < 12u ? jn : 11u];
        push_darts(more, op + kGolden, x.x + (1u << 26), x.y, x.z, x.w, lo);
    };

    for (int64_t tile = first; tile < end;) {
        // segment: geometry and key of up to kSegTiles tiles; elements sorted by nu_top (descending)
        __syncwarp();
        int nut[kSegTiles];
        uint64_t et[kSegTiles];
        uint32_t vt[kSegTiles], rank[kSegTiles];
#pragma unroll
        for (int t = 0; t < kSegTiles; ++t) {
            nut[t] = -1;
            et[t] = 0;
            vt[t] = 0;
            rank[t] = 0;
            if (tile < end) {
                const int64_t pos = tile + lane;
                uint64_t F = 0;
                if (pos < end) {
                    nut[t] = weight_geometry(__float_as_uint(p.weights[pos]), p.t, F, escale);
                    if (nut[t] >= 0) et[t] = mix64(p.sigma + kGolden * ((uint64_t)p.indices[pos] + 1));
                }
                if (__any_sync(kFull, nut[t] == -2)) return DM_ERANGE;
                if (!__all_sync(kFull, nut[t] <= 31)) return kDefer;
                vt[t] = (uint32_t)(F >> 40);
                tile += stride;
            }
        }
        int nhi = -1, nlo = 32;
#pragma unroll
        for (int t = 0; t < kSegTiles; ++t) {
            nhi = max(nhi, nut[t]);
            if (nut[t] >= 0) nlo = min(nlo, nut[t]);
        }
        nhi = __reduce_max_sync(kFull, nhi);
        nlo = __reduce_min_sync(kFull, nlo);
        if (nhi < 0) continue;
        // ranks in descending nu_top order; lane v keeps cnt(v), the elements with nu_top >= v
        uint32_t placed = 0, mycnt = 0;
        for (int v = nhi; v >= nlo; --v) {
#pragma unroll
            for (int t = 0; t < kSegTiles; ++t) {
                const unsigned mv = __ballot_sync(kFull, nut[t] == v);
                if (nut[t] == v) rank[t] = placed + __popc(mv & lt);
                placed += __popc(mv);
            }
            if (lane == v) mycnt = placed;
        }
        if (lane < nlo) mycnt = placed;
#pragma unroll
        for (int t = 0; t < kSegTiles; ++t)
            if (nut[t] >= 0 && DM_EXPECT(rank[t] < (uint32_t)kSeg))
                *reinterpret_cast<uint4 *>(&m.el[rank[t]]) =
                    make_uint4((uint32_t)et[t], (uint32_t)(et[t] >> 32), 0u, vt[t] | ((uint32_t)nut[t] << 24));
        // region nu = lane holds cnt(nu) rows(nu) areas; C(nu) is their offset in the segment
        const uint64_t A = (uint64_t)mycnt * myrows;
        const uint64_t incl = warp_incl_scan(A, lane);
        const uint64_t base = __shfl_sync(kFull, incl, 31);
        if (base >= (1ull << 31)) return kDefer;
        m.rb[lane].cnt = mycnt;
        m.rb[lane].C = (uint32_t)(incl - A);
        __syncwarp();
        const uint32_t total = (uint32_t)base, lanes = 32u * (uint32_t)nparts;
        const uint32_t share = (total + lanes - 1) / lanes;
        const uint32_t lo = share * (32u * (uint32_t)part + (uint32_t)lane);
        uint32_t left = lo < total ? min(share, total - lo) : 0u;
        // area steps of this warp: lane 0 has the largest share
        const uint32_t lo0 = share * 32u * (uint32_t)part;
        const uint32_t steps = lo0 < total ? min(share, total - lo0) : 0u;
        WalkF s{};
        if (left) s.locate(lo, m);
        for (uint32_t st = 0; st < steps; ++st) {
            // area step: X >= 1 and X >= 2 decide the first dart and the dart queue; the count
            // itself is resolved dart by dart from the Poisson uniform ua
            const bool act = left != 0;
            const uint64_t a = mix64(s.ctr);
            const uint32_t ua = (uint32_t)(a >> 32);
            const bool x1 = act && ua >= c_pois[0], x2 = act && ua >= c_pois[1];
            const uint32_t uthr = s.r + 1 == s.rhi ? s.lastthr : (1u << 25);
            const uint32_t ulo = LOWER && s.r == s.rlo ? s.firstlo : 0u;
            const uint64_t d = mix64(a + kGolden);
            const uint32_t u = (uint32_t)(d >> 40), vv = (uint32_t)(d >> 16) & kUMask;
            bool keep = x1 && u < uthr && vv <= s.vmax;
            if constexpr (LOWER) keep = keep && u >= ulo;
            if (COUNT) { cnt[0] += act; cnt[1] += act ? (uint32_t)poisson1(ua, c_pois) : 0u; }
            push_kept(keep, d, s.r, (uint32_t)s.nu);
            push_darts(x2, a + 2 * kGolden, uthr | (1u << 26), s.vmax | ((uint32_t)s.nu << 24), s.r, ua, ulo);
            if (act && --left) s.advance(m);
            // serve the full queues: each holds fewer than 32 entries before an area step, so
            // fewer than 64 after it, and fewer than 32 again once served
            while (((kt - kh) | (xt - xh)) >= 32u) {
                if (kt - kh >= 32u) kept_step(32u);
                else dart_step(32u);
            }
        }
    }
    for (;;) {                                    // drain both queues
        if (kt - kh >= 32u) kept_step(32u);
        else if (xt != xh) dart_step(min(xt - xh, 32u));
        else if (kt != kh) kept_step(kt - kh);
        else break;
    }
    __syncwarp();
    return 0;
}

// ==========================================================================================
// General path: every region (nu, rho), columns w and rows r, in 64-bit arithmetic, with the
// same three kinds of warp-wide steps as the fast path (area steps with the area's first dart,
// dart steps over queued areas, bucket steps over queued kept darts).  A dart of an area has
// rank (pb + (u << sh)) 2^-S with the area's rank base pb (a multiple of 2^24), sh = 38 - nu and
// S = 62 - rho, and hits x iff v <= vmax; pv = pb + vmax holds both.  A dart is kept iff its
// binary32 rank code lies in [bits(theta_{p-1}), bits(theta_p)) (the lower bound only for the
// sinks that must not see a dart twice).
// ==========================================================================================
struct GenMem {
    uint64_t *te, *tF, *toff;
    int *tnu;
    uint4 *kq;                          // kept queue [kQ]: dart hash (low, high word), rank code, unused
    uint4 *xa;                          // dart queue [kQ]: counter of the area's dart j (low, high), pv (low, high)
    uint2 *xb;                          // dart queue [kQ]: j | nu << 4 | rho << 10, the area's Poisson uniform
};

constexpr size_t kGenPathBytes = 3 * 32 * 8 + 32 * 4 + (size_t)kQ * (16 + 16 + 8);
static_assert((3 * 32 * 8 + 32 * 4) % 16 == 0, "general-path queues keep 16-byte alignment");

__device__ __forceinline__ GenMem carve_gen(unsigned char *base) {
    GenMem m;
    m.te = reinterpret_cast<uint64_t *>(base);
    m.tF = m.te + 32;
    m.toff = m.tF + 32;
    m.tnu = reinterpret_cast<int *>(m.toff + 32);
    m.kq = reinterpret_cast<uint4 *>(m.tnu + 32);
    m.xa = m.kq + kQ;
    m.xb = reinterpret_cast<uint2 *>(m.xa + kQ);
    return m;
}

__device__ __forceinline__ int tile_element(const GenMem &m, uint64_t idx) {
    int el = 0;                               // last element whose offset is <= idx
#pragma unroll
    for (int step = 16; step; step >>= 1) {
        int c = el + step;
        if (c < 32 && m.toff[c] <= idx) el = c;
    }
    return el;
}

// sum_{nu=1..m} floor(G / 2^(64 - nu)) = 2H - popc(H) with H = floor(G / 2^(64 - m)); 0 for m = 0.
__device__ __forceinline__ uint64_t floor_sum(uint64_t G, int m) {
    if (m <= 0) return 0;
    const uint64_t H = G >> (64 - m);
    return 2 * H - (uint64_t)__popcll(H);
}

// Rows of rank region rho summed over weight regions nu = 0 .. n-1 (every one of them below the
// element's last region, so all its columns count): sum of rows_hi - rows_lo in closed form.
__device__ __forceinline__ uint64_t rows_upto(const PassCut &pc, int rho, int n) {
    if (n <= 0) return 0;
    uint64_t hi = rho == pc.rho_top ? (uint64_t)n + floor_sum(pc.gm1, n - 1) : (1ull << n) - 1;
    uint64_t lo = rho == pc.rho_lo ? floor_sum(pc.gfl_lo, n - 1) : 0;
    return hi - lo;
}

struct WalkG {
    int el, nu, rho, nutop;
    uint64_t w, r, ncols, rlo, rhi;
    uint64_t e, F, WT, rbase, packhi, ctr;

    // areas of weight regions nu < n (n <= nutop): 2^rho columns each
    __device__ static uint64_t count_below(int n, const PassCut &pc) {
        uint64_t total = 0;
        for (int h = pc.rho_lo; h <= pc.rho_top; ++h) total += rows_upto(pc, h, n) << h;
        return total;
    }
    // areas of the last weight region nu = nutop
    __device__ static uint64_t count_top(int nutop, uint64_t F, const PassCut &pc) {
        uint64_t total = 0;
        for (int h = pc.rho_lo; h <= pc.rho_top; ++h)
            total += cols(nutop, h, nutop, F) * (rows_hi(pc, nutop, h) - rows_lo(pc, nutop, h));
        return total;
    }
    __device__ static uint64_t count(int nutop, uint64_t F, const PassCut &pc) {
        return count_below(nutop, pc) + count_top(nutop, F, pc);
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
    __device__ void load(const GenMem &m) {
        if (!DM_EXPECT(el >= 0 && el < 32)) el = 0;
        e = m.te[el];
        F = m.tF[el];
        nutop = m.tnu[el];
    }
    __device__ void locate(uint64_t idx, const GenMem &m, const PassCut &pc) {
        el = tile_element(m, idx);
        load(m);
        uint64_t li = idx - m.toff[el];
        // weight region: the largest n <= nutop with count_below(n) <= li (binary search;
        // count_below is non-decreasing in n)
        int lo = 0, hi = nutop;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (count_below(mid, pc) <= li) lo = mid;
            else hi = mid - 1;
        }
        nu = lo;
        li -= count_below(nu, pc);
        for (rho = pc.rho_lo; rho <= pc.rho_top; ++rho) {
            region(pc);
            const uint64_t nrows = rhi - rlo, c = ncols * nrows;
            if (li < c) {
                w = li / nrows;
                r = rlo + (li - w * nrows);
                break;
            }
            li -= c;
        }
        set_ctr();
    }
    __device__ uint64_t pv() const {
        return rbase + (r << (62 - nu)) + min(WT - (w << 24), (uint64_t)kUMask);
    }
    __device__ void advance(const GenMem &m, const PassCut &pc) {
        ++r;
        ctr += kGolden;
        if (r < rhi) return;
        if (++w < ncols) {
            // next column of the region: its row rlo is (2^nu - rhi + rlo) counter steps on
            // (the pack holds w 2^nu + r with r < 2^nu)
            r = rlo;
            ctr += kGolden * ((1ull << nu) + rlo - rhi);
            return;
        }
        w = 0;
        if (++rho > pc.rho_top) {
            rho = pc.rho_lo;
            if (++nu > nutop) {
                nu = 0;
                do { ++el; } while (el < 32 && m.tnu[el] < 0);
                if (el >= 32) return;             // past the tile: the lane is done
                load(m);
            }
        }
        region(pc);
        r = rlo;
        set_ctr();
    }
};

// One pass with the general walk over tiles first, first + stride, ... of the row [.., end), each
// tile's areas split among nparts warps (this one is number part).  Returns 0 or an error code.
template <class Sink, bool COUNT>
__device__ int gen_pass(const SketchParams &p, int64_t first, int64_t stride, int64_t end, const PassCut &pc,
                        const GenMem &m, Sink &sink, int lane, unsigned long long *cnt, int escale = 0,
                        int part = 0, int nparts = 1) {
    constexpr bool LOWER = Sink::kLowerCut;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t kh = 0, kt = 0, xh = 0, xt = 0;     // kept and dart queues: heads and tails

    // binary32 code of rank = P 2^-S rounded toward zero: exact u64 -> f32 conversion in
    // round-toward-zero mode, then the exponent lowered by S; kept iff in the pass's code range
    auto rank_code = [](uint64_t P, uint32_t S) -> uint32_t {
        return P ? __float_as_uint(__ull2float_rz(P)) - (S << 23) : 0u;
    };
    auto in_band = [&](uint32_t code) -> bool {
        if constexpr (LOWER) return code < pc.cthr && code >= pc.cthr_lo;
        return code < pc.cthr;
    };
    auto push_kept = [&](bool keep, uint64_t d, uint32_t code) {
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) m.kq[(kt + __popc(km & lt)) & (kQ - 1)] = make_uint4((uint32_t)d, (uint32_t)(d >> 32), code, 0u);
        kt += __popc(km);
        (void)DM_EXPECT(kt - kh <= (uint32_t)kQ);
        if (COUNT && keep) cnt[2]++;
    };
    auto push_darts = [&](bool more, uint64_t op, uint64_t pv, uint32_t w, uint32_t ua) {
        const unsigned xm = __ballot_sync(kFull, more);
        if (more) {
            const uint32_t i = (xt + __popc(xm & lt)) & (kQ - 1);
            m.xa[i] = make_uint4((uint32_t)op, (uint32_t)(op >> 32), (uint32_t)pv, (uint32_t)(pv >> 32));
            m.xb[i] = make_uint2(w, ua);
        }
        xt += __popc(xm);
        (void)DM_EXPECT(xt - xh <= (uint32_t)kQ);
    };
    // bucket step over the n (<= 32) oldest kept darts
    auto kept_step = [&](uint32_t n) {
        __syncwarp();
        const bool v = (uint32_t)lane < n;
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        if (v) q = m.kq[(kh + (uint32_t)lane) & (kQ - 1)];
        kh += n;
        const uint64_t h = mix64((((uint64_t)q.y << 32) | q.x) ^ kSlotSalt);
        sink.put_batch(v, h, q.z, lane);
        __syncwarp();
    };
    // dart step over the n (<= 32) oldest queued areas: dart j of each; the area goes back to
    // the queue when dart j + 1 exists (its Poisson uniform reaches T[j + 1])
    auto dart_step = [&](uint32_t n) {
        __syncwarp();
        const bool v = (uint32_t)lane < n;
        uint4 xa = make_uint4(0u, 0u, 0u, 0u);
        uint2 xb = make_uint2(0u, 0u);
        if (v) {
            const uint32_t i = (xh + (uint32_t)lane) & (kQ - 1);
            xa = m.xa[i];
            xb = m.xb[i];
        }
        xh += n;
        __syncwarp();                             // every lane has read its entry before any push
        const uint64_t op = ((uint64_t)xa.y << 32) | xa.x, pv = ((uint64_t)xa.w << 32) | xa.z;
        const uint64_t d = mix64(op);
        const uint32_t u = (uint32_t)(d >> 40), vv = (uint32_t)(d >> 16) & kUMask;
        const uint32_t nu = (xb.x >> 4) & 63u, rho = (xb.x >> 10) & 63u;
        const uint32_t code = rank_code((pv & ~(uint64_t)kUMask) + ((uint64_t)u << (38u - nu)), 62u - rho);
        push_kept(v && vv <= ((uint32_t)pv & kUMask) && in_band(code), d, code);
        const uint32_t jn = (xb.x & 15u) + 1u;
        const bool more = v && jn < 12u && xb.y >= c_pois[jn < 12u ? jn : 11u];
        push_darts(more, op + kGolden, pv, xb.x + 1u, xb.y);
    };

    for (int64_t tile = first; tile < end; tile += stride) {
        const int64_t pos = tile + lane;
        int nutop = -1;
        uint64_t F = 0, e = 0;
        if (pos < end) {
            nutop = weight_geometry(__float_as_uint(p.weights[pos]), p.t, F, escale);
            if (nutop >= 0) e = mix64(p.sigma + kGolden * ((uint64_t)p.indices[pos] + 1));
        }
        if (__any_sync(kFull, nutop == -2)) return DM_ERANGE;
        const uint64_t n_el = nutop >= 0 ? WalkG::count(nutop, F, pc) : 0;
        const uint64_t incl = warp_incl_scan(n_el, lane);
        __syncwarp();
        m.te[lane] = e;
        m.tF[lane] = F;
        m.tnu[lane] = n_el ? nutop : -1;
        m.toff[lane] = incl - n_el;
        __syncwarp();
        const uint64_t total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        const uint64_t lanes = 32ull * (uint64_t)nparts;
        const uint64_t share = (total + lanes - 1) / lanes;
        const uint64_t lo = share * (32ull * (uint64_t)part + (uint64_t)lane);
        uint64_t left = lo < total ? min(share, total - lo) : 0;   // areas of this lane
        const uint64_t lo0 = share * 32ull * (uint64_t)part;        // lane 0 has the largest share
        const uint64_t steps = lo0 < total ? min(share, total - lo0) : 0;
        WalkG s{};
        if (left) s.locate(lo, m, pc);
        for (uint64_t st = 0; st < steps; ++st) {
            // area step: X >= 1 and X >= 2 from the Poisson uniform ua; the first dart at once
            const bool act = left != 0;
            const uint64_t a = mix64(s.ctr);
            const uint32_t ua = (uint32_t)(a >> 32);
            const bool x1 = act && ua >= c_pois[0], x2 = act && ua >= c_pois[1];
            const uint64_t pv = s.pv();
            const uint64_t d = mix64(a + kGolden);
            const uint32_t u = (uint32_t)(d >> 40), vv = (uint32_t)(d >> 16) & kUMask;
            const uint32_t code = rank_code((pv & ~(uint64_t)kUMask) + ((uint64_t)u << (38 - s.nu)),
                                            62u - (uint32_t)s.rho);
            if (COUNT) { cnt[0] += act; cnt[1] += act ? (uint32_t)poisson1(ua, c_pois) : 0u; }
            push_kept(x1 && vv <= ((uint32_t)pv & kUMask) && in_band(code), d, code);
            push_darts(x2, a + 2 * kGolden, pv, 1u | ((uint32_t)s.nu << 4) | ((uint32_t)s.rho << 10), ua);
            if (act && --left) s.advance(m, pc);
            while (((kt - kh) | (xt - xh)) >= 32u) {   // serve the full queues (as in the fast pass)
                if (kt - kh >= 32u) kept_step(32u);
                else dart_step(32u);
            }
        }
    }
    for (;;) {                                    // drain both queues
        if (kt - kh >= 32u) kept_step(32u);
        else if (xt != xh) dart_step(min(xt - xh, 32u));
        else if (kt != kh) kept_step(kt - kh);
        else break;
    }
    __syncwarp();
    return 0;
}

// ==========================================================================================
// Kernel.  MODE 0 (fast): sets in order; passes with a limit >= 1, and tiles outside the
// 32-bit walk, send the set to the queue.  MODE 1 (general): sets from the queue, every pass
// with the general walk.  Warps are persistent and claim work items from a global counter.
// ==========================================================================================
// Visits the weights w[beg, end) of a row with n threads (this one is number i < n): 128-bit
// loads over the row's 16-byte-aligned middle, 32-bit loads for the at most three weights before
// it and three after it.  Each weight is visited by exactly one thread, in no particular order.
template <class F>
__device__ __forceinline__ void for_row_weights(const float *w, int64_t beg, int64_t end, int i, int n, F &&f) {
    const float *row = w + beg;
    const int64_t len = end - beg;
    const uint32_t mis = (uint32_t)reinterpret_cast<uintptr_t>(row) & 15u;
    int64_t head = (mis & 3u) ? len : (int64_t)(((16u - mis) & 15u) >> 2);   // a float* is 4-byte aligned
    if (head > len) head = len;
    const int64_t nv = (len - head) >> 2;
    for (int64_t j = i; j < head; j += n) f(row[j]);
    const float4 *v = reinterpret_cast<const float4 *>(row + head);
    for (int64_t j = i; j < nv; j += n) {
        const float4 q = v[j];
        f(q.x);
        f(q.y);
        f(q.z);
        f(q.w);
    }
    for (int64_t j = head + 4 * nv + i; j < len; j += n) f(row[j]);
}

template <class Sink, bool BBIT, bool COUNT, int MODE>
__global__ void __launch_bounds__(256, MODE == 0 ? 4 : 3) set_kernel(const SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)wib * (MODE == 0 ? p.warp_bytes_fast : p.warp_bytes);
    Sink sink;
    sink.bind(wbase, p);
    const FastMem fm = carve_fast(wbase + p.sink_bytes);
    const GenMem gm = carve_gen(wbase + p.sink_bytes);
    // general kernel: the queued sets [w0, n_work) (see gen_part); fast kernel: the fast sets of
    // the batched form, or every set
    const int64_t w0 = MODE == 1 && p.gen_part == 2 ? (int64_t)p.hist[kTotals + 1] : 0;
    const int64_t n_work = MODE == 1 ? (p.gen_part == 1 ? (int64_t)p.hist[kTotals + 1] : (int64_t)*p.queue_count)
                                     : (p.sched == 2 ? (int64_t)p.hist[kTotals] : p.n_sets);
    unsigned int *next = MODE == 1 && p.gen_part == 2 ? p.hist + kDeferNext : p.work_next + MODE;
    const int64_t static_wi = (int64_t)blockIdx.x * p.warps_per_block + wib;
    for (int round = 0;; ++round) {
        int64_t wi;
        if (p.sched == 1) {                        // plain form: one set per warp
            if (round) break;
            wi = static_wi;
        } else {
            unsigned int c = 0;
            if (lane == 0) c = atomicAdd(next, 1u);
            wi = w0 + (int64_t)__shfl_sync(kFull, c, 0);
        }
        if (wi >= n_work) break;
        const int64_t set = MODE == 1 ? (int64_t)p.queue[wi] : (p.sched == 2 ? (int64_t)p.order[wi] : wi);
        const int64_t beg = p.indptr[set], end = p.indptr[set + 1];
        // ||x||_1 and input validation
        float l1 = 0.f;
        bool bad = false;
        for_row_weights(p.weights, beg, end, lane, 32, [&](float x) {
            if (!(x >= 0.f) || isinf(x)) bad = true;
            else l1 += x;
        });
#pragma unroll
        for (int o = 16; o; o >>= 1) l1 += __shfl_xor_sync(kFull, l1, o);
        int err = __any_sync(kFull, bad) ? DM_EINVAL : 0;
        sink.set_row(p, set);
        sink.reset(lane);
        unsigned long long cnt[3] = {0, 0, 0};
        unsigned long long passes = 0;
        bool deferred = false;
        const int sc = p.scale ? p.scale[set] : 0;
        if (!err && l1 > 0.f) {
            // first limit phi0 / (|x|_1 2^sc); any positive value gives the same result
            uint32_t th = __float_as_uint(sc ? scalbnf(__fdiv_rn(p.phi0, l1), -sc) : __fdiv_rn(p.phi0, l1));
            PassCut pc;
            pc.rho_lo = 0;
            pc.gfl_lo = 0;
            pc.cthr_lo = 0;
            for (int pass = 0;; ++pass) {
                if (pass == kMaxPasses) { err = DM_EOVERFLOW; break; }
                RankCut rc;
                if (!rank_cut(th, rc)) { err = DM_ERANGE; break; }
                pc.rho_top = rc.rho_top;
                pc.gm1 = rc.gm1;
                pc.cthr = th;
                if (MODE == 0 && pc.rho_top != 0) { deferred = true; break; }
                err = MODE == 0 ? fast_pass<Sink, COUNT>(p, beg, 32, end, pc, fm, sink, lane, cnt, sc)
                                : gen_pass<Sink, COUNT>(p, beg, 32, end, pc, gm, sink, lane, cnt, sc);
                ++passes;
                if (err == kDefer) { err = 0; deferred = true; break; }
                if (err) break;
                if (sink.filled(lane)) break;
                // next band starts where this limit ended
                pc.rho_lo = rc.g_one ? rc.rho_top + 1 : rc.rho_top;
                pc.gfl_lo = rc.g_one ? 0 : rc.gfl;
                pc.cthr_lo = th;
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
            sink.clear_to_error(lane);
        }
        sink.template finish<BBIT>(p, set, err != 0, lane);
        __syncwarp();
    }
}

// ==========================================================================================
// Batched form.  classify: per set, class (0 fast: first limit below 1; 1 general; 2 large:
// >= large_nnz elements or a work estimate >= large_work, sketches only) and a size bin that
// sorts costlier sets first:
// bin = 31 - floor(log2(E)) with E the Lemma 2 estimate of the areas inspected at the first
// limit theta = phi0 / |x|_1,
//     E = phi0 t + sum_i (log2(1 + t x_i) + 1) + nnz log2(1 + theta)
// (the linear term, then per element the weight regions and the rank regions).  scan: bin
// offsets per class; scatter: fast sets to order[0..nF), general sets to queue[0..nG) (the
// general kernel's list; the fast kernel appends the sets it defers after them), large sets to
// order[nF..nF+nL).  The estimate only orders work; it never changes a result.
// ==========================================================================================
__global__ void __launch_bounds__(256) classify_kernel(const SketchParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const float t = (float)p.t;
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < p.n_sets; s += nw) {
        const int64_t beg = p.indptr[s], end = p.indptr[s + 1], nnz = end - beg;
        float l1 = 0.f, wlog = 0.f;
        for_row_weights(p.weights, beg, end, lane, 32, [&](float x) {
            l1 += x;
            if (x > 0.f) wlog += __log2f(1.0f + t * x) + 1.0f;
        });
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            l1 += __shfl_xor_sync(kFull, l1, o);
            wlog += __shfl_xor_sync(kFull, wlog, o);
        }
        if (lane == 0) {
            float est = 1.0f;
            if (l1 > 0.f && l1 < 3.0e38f && wlog < 3.0e38f)
                est += p.phi0 * t + wlog + (float)nnz * __log2f(1.0f + p.phi0 / l1);
            int c;
            if (p.large_nnz > 0 && nnz >= p.large_nnz) c = 2;
            else if (p.large_work > 0.f && nnz > 0 && est >= p.large_work) c = 2;
            else c = (!(l1 > 0.f) || scalbnf(__fdiv_rn(p.phi0, l1), p.scale ? -p.scale[s] : 0) < 1.0f) ? 0 : 1;
            // floor(log2(est)) from the exponent field (est >= 1, finite or +inf)
            int lg = (int)((__float_as_uint(est) >> 23) & 0xFFu) - 127;
            const int bin = 31 - (lg > 31 ? 31 : lg);
            p.cls[s] = (uint8_t)(c * kBins + (bin < 0 ? 0 : bin));
            atomicAdd(&p.hist[c * kBins + (bin < 0 ? 0 : bin)], 1u);
        }
    }
}

// Weight class c = floor(log2 |x|_1) per set (Section 3's split of the data into classes
// |x|_1 in [2^c, 2^(c+1))), where |x|_1 is the exact sum of the set's positive finite binary32
// weights (zero, negative, NaN and infinite weights take no part).  A weight is M 2^(s - 149) with
// M < 2^24 and s = max(exponent field, 1) - 1 in [0, 253], so N = |x|_1 2^149 = sum M 2^s is an
// integer.  Each lane adds its elements' M 2^s into nine base-2^32 digits, each held in a 64-bit
// word of a shared-memory column of its own (the upper halves collect carries); the warp then
// sums the columns digit by digit, propagates the carries and takes the class from the highest
// set bit, c = bitlen(N) - 1 - 149.  Every step is integer addition, so the result does not
// depend on the order of the elements.  Rows must have fewer than 2^32 elements.
constexpr int kClassDigits = 9;         // digits of the per-lane sums: bits 0 .. 287
constexpr int kClassWarps = 8;

__global__ void __launch_bounds__(32 * kClassWarps) weight_class_kernel(const int64_t *indptr, const float *weights,
                                                                        int64_t n_sets, int32_t *out,
                                                                        int32_t *scale_out, int32_t norm_exp) {
    __shared__ uint64_t acc[kClassWarps][kClassDigits][32];      // [warp][digit][lane]
    __shared__ uint64_t tot[kClassWarps][kClassDigits];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * kClassWarps;
    for (int64_t s = (int64_t)blockIdx.x * kClassWarps + wid; s < n_sets; s += nw) {
#pragma unroll
        for (int d = 0; d < kClassDigits; ++d) acc[wid][d][lane] = 0;
        for_row_weights(weights, indptr[s], indptr[s + 1], lane, 32, [&](float x) {
            const uint32_t xb = __float_as_uint(x), ex = xb >> 23;
            if (xb == 0 || ex >= 255u) return;            // zero, negative (sign bit set), NaN or infinite
            const uint32_t M = ex ? (xb & 0x7FFFFFu) | 0x800000u : xb;
            const uint32_t sh = (ex ? ex : 1u) - 1u;
            const uint64_t v = (uint64_t)M << (sh & 31u);   // below 2^55: digits sh / 32 and sh / 32 + 1
            const uint32_t d = sh >> 5;
            acc[wid][d][lane] += (uint32_t)v;
            acc[wid][d + 1][lane] += v >> 32;
        });
        __syncwarp();
        if (lane < kClassDigits) {                       // digit sums over the 32 columns
            uint64_t t = 0;
            for (int j = 0; j < 32; ++j) t += acc[wid][lane][j];
            tot[wid][lane] = t;
        }
        __syncwarp();
        if (lane == 0) {
            uint64_t carry = 0;
            int c = 0;
            for (int d = 0; d <= kClassDigits; ++d) {   // one more digit for the last carry
                const uint64_t word = (d < kClassDigits ? tot[wid][d] : 0ull) + carry;
                const uint32_t digit = (uint32_t)word;
                carry = word >> 32;
                if (digit) c = 32 * d + (31 - __clz(digit)) - 149;
            }
            if (out) out[s] = c;
            if (scale_out) scale_out[s] = norm_exp - c;
        }
        __syncwarp();
    }
}

__global__ void scan_kernel(const SketchParams p) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int c = 0; c < kClasses; ++c) {
        unsigned int off = 0;
        for (int b = 0; b < kBins; ++b) {
            p.hist[kCursors + c * kBins + b] = off;
            off += p.hist[c * kBins + b];
        }
        p.hist[kTotals + c] = off;
    }
    *p.queue_count = p.hist[kTotals + 1];
}

__global__ void __launch_bounds__(256) scatter_kernel(const SketchParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.n_sets; s += stride) {
        const int cb = p.cls[s], c = cb / kBins;
        const unsigned int pos = atomicAdd(&p.hist[kCursors + cb], 1u);
        if (c == 0) p.order[pos] = (int32_t)s;
        else if (c == 1) p.queue[pos] = (int32_t)s;
        else p.order[p.hist[kTotals] + pos] = (int32_t)s;
    }
}

// Large sets: a block per set.  The block's warps share the set's k bucket minima in shared
// memory (the shared-memory minimum works across warps).  A set of at least two tiles per warp
// has its tiles dealt round-robin to the warps; a smaller one (few elements, much work) has every tile's
// areas split among all the warps.  Passes are separated by block barriers.  A pass runs the
// fast walk when the limit is below 1 and every tile allows it, else the general walk over all
// tiles (a dart seen twice does not change a minimum).
size_t large_block_bytes(int k, int warps, bool key_row) {
    const size_t per = kFastPathBytes > kGenPathBytes ? kFastPathBytes : kGenPathBytes;
    return sketch_sink_bytes(k, key_row) + (size_t)warps * per + 64;
}

template <class Sink, bool BBIT, bool COUNT>
__global__ void __launch_bounds__(256, 2) large_kernel(const SketchParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const size_t per = kFastPathBytes > kGenPathBytes ? kFastPathBytes : kGenPathBytes;
    Sink sink;
    sink.bind(smem, p);
    unsigned char *wbase = smem + sketch_sink_bytes(p.k, p.key_row != 0) + (size_t)wid * per;
    const FastMem fm = carve_fast(wbase);
    const GenMem gm = carve_gen(wbase);
    int *flags = reinterpret_cast<int *>(smem + sketch_sink_bytes(p.k, p.key_row != 0) + (size_t)nwarps * per);
    float *wsum = reinterpret_cast<float *>(flags + 4);
    const int64_t n_work = p.hist[kTotals + 2], base = p.hist[kTotals];
    for (;;) {
        if (threadIdx.x == 0) flags[0] = (int)atomicAdd(p.work_next + 2, 1u);
        __syncthreads();
        const int64_t wi = flags[0];
        if (wi >= n_work) break;
        const int64_t set = p.order[base + wi];
        const int64_t beg = p.indptr[set], end = p.indptr[set + 1];
        const bool split = end - beg < 64 * (int64_t)nwarps;
        float l1 = 0.f;
        int bad = 0;
        for_row_weights(p.weights, beg, end, (int)threadIdx.x, (int)blockDim.x, [&](float x) {
            if (!(x >= 0.f) || isinf(x)) bad = 1;
            else l1 += x;
        });
#pragma unroll
        for (int o = 16; o; o >>= 1) l1 += __shfl_xor_sync(kFull, l1, o);
        if (lane == 0) wsum[wid] = l1;
        sink.set_row(p, set);
        if (wid == 0) sink.reset(lane);
        int err = __syncthreads_or(bad) ? DM_EINVAL : 0;
        l1 = 0.f;
        for (int w = 0; w < nwarps; ++w) l1 += wsum[w];
        unsigned long long cnt[3] = {0, 0, 0};
        unsigned long long passes = 0;
        const int sc = p.scale ? p.scale[set] : 0;
        if (!err && l1 > 0.f) {
            uint32_t th = __float_as_uint(sc ? scalbnf(__fdiv_rn(p.phi0, l1), -sc) : __fdiv_rn(p.phi0, l1));
            PassCut pc;
            pc.rho_lo = 0;
            pc.gfl_lo = 0;
            pc.cthr_lo = 0;
            for (int pass = 0;; ++pass) {
                if (pass == kMaxPasses) { err = DM_EOVERFLOW; break; }
                RankCut rc;
                if (!rank_cut(th, rc)) { err = DM_ERANGE; break; }
                pc.rho_top = rc.rho_top;
                pc.gm1 = rc.gm1;
                pc.cthr = th;
                int e = kDefer;
                if (pc.rho_top == 0)
                    e = split ? fast_pass<Sink, COUNT>(p, beg, 32, end, pc, fm, sink, lane, cnt, sc, wid, nwarps)
                              : fast_pass<Sink, COUNT>(p, beg + 32 * wid, 32 * nwarps, end, pc, fm, sink, lane, cnt, sc);
                const int any_defer = __syncthreads_or(e == kDefer);
                if (any_defer)
                    e = split ? gen_pass<Sink, COUNT>(p, beg, 32, end, pc, gm, sink, lane, cnt, sc, wid, nwarps)
                              : gen_pass<Sink, COUNT>(p, beg + 32 * wid, 32 * nwarps, end, pc, gm, sink, lane, cnt, sc);
                ++passes;
                if (__syncthreads_or(e == DM_ERANGE)) { err = DM_ERANGE; break; }
                int empty = 0;
                for (uint32_t j = threadIdx.x; j < (uint32_t)p.k; j += blockDim.x) empty |= sink.empty_bucket(j);
                if (!__syncthreads_or(empty)) break;
                pc.rho_lo = rc.g_one ? rc.rho_top + 1 : rc.rho_top;
                pc.gfl_lo = rc.g_one ? 0 : rc.gfl;
                pc.cthr_lo = th;
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
            if (threadIdx.x == 0 && p.counters) atomicAdd(&p.counters[3], passes);
        }
        __syncthreads();
        if (wid == 0) {
            if (err) {
                if (lane == 0) set_status(p.status, err);
                sink.clear_to_error(lane);
            }
            sink.template finish<BBIT>(p, set, err != 0, lane);
        }
        __syncthreads();
    }
}

template <bool BBIT, bool COUNT>
static cudaError_t launch_large(const SketchParams &p, int grid, cudaStream_t st) {
    const size_t smem = large_block_bytes(p.k, p.large_warps, p.key_row != 0);
    if (p.key_row) large_kernel<RowSink, BBIT, COUNT><<<grid, 32 * p.large_warps, smem, st>>>(p);
    else large_kernel<SketchSink, BBIT, COUNT><<<grid, 32 * p.large_warps, smem, st>>>(p);
    return cudaGetLastError();
}

int large_blocks_per_sm(bool bbit, int warps, size_t smem, bool key_row) {
    const void *fn = key_row ? (bbit ? (const void *)large_kernel<RowSink, true, false>
                                     : (const void *)large_kernel<RowSink, false, false>)
                             : (bbit ? (const void *)large_kernel<SketchSink, true, false>
                                     : (const void *)large_kernel<SketchSink, false, false>);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * warps, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_weight_classes(const int64_t *indptr, const float *weights, int64_t n_sets, int32_t *out,
                                  int32_t *scale_out, int32_t norm_exp, int sm_count, cudaStream_t st) {
    const int64_t blocks = (n_sets + 7) / 8, cap = 16LL * (sm_count > 0 ? sm_count : 1);
    weight_class_kernel<<<(int)(blocks < cap ? blocks : cap), 32 * kClassWarps, 0, st>>>(indptr, weights, n_sets, out,
                                                                                          scale_out, norm_exp);
    return cudaGetLastError();
}

size_t call_scratch_bytes(int64_t n_sets) {
    const size_t a = ((size_t)n_sets * 4 + 255) / 256 * 256, c = ((size_t)n_sets + 255) / 256 * 256;
    return 2 * a + c + kHeaderBytes;
}

void carve_call_scratch(void *base, int64_t n_sets, SketchParams &p) {
    const size_t a = ((size_t)n_sets * 4 + 255) / 256 * 256, c = ((size_t)n_sets + 255) / 256 * 256;
    char *b = (char *)base;
    p.queue = (int32_t *)b;
    p.order = (int32_t *)(b + a);
    p.cls = (uint8_t *)(b + 2 * a);
    p.queue_count = (unsigned int *)(b + 2 * a + c);
    p.work_next = p.queue_count + 1;
    p.hist = p.queue_count + 4;
}

// Checked build: the source line of the first failed index check since the last call (0:
// none), cleared on reading.  The product build has no checks and returns 0.
cudaError_t take_check_line(int *line, cudaStream_t st) {
    *line = 0;
#ifdef DM_CHECKED
    cudaError_t e = cudaMemcpyFromSymbolAsync(line, g_dm_check, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && *line) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_dm_check, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
#else
    (void)st;
    return cudaSuccess;
#endif
}

cudaError_t upload_poisson_table(const uint32_t *T) {
    return cudaMemcpyToSymbol(c_pois, T, 12 * sizeof(uint32_t));
}

template <class Sink, bool BBIT, bool COUNT, int MODE>
static const void *kernel_fn() {
    return (const void *)set_kernel<Sink, BBIT, COUNT, MODE>;
}

template <class Sink, bool BBIT, bool COUNT, int MODE>
static cudaError_t launch_t(const SketchParams &p, int grid, cudaStream_t st) {
    const size_t smem = (size_t)(MODE == 0 ? p.warp_bytes_fast : p.warp_bytes) * p.warps_per_block;
    set_kernel<Sink, BBIT, COUNT, MODE><<<grid, 32 * p.warps_per_block, smem, st>>>(p);
    return cudaGetLastError();
}

template <class Sink, int MODE>
static cudaError_t launch_mode(const SketchParams &p, bool bbit, bool count, int grid, cudaStream_t st) {
    if (bbit) return count ? launch_t<Sink, true, true, MODE>(p, grid, st) : launch_t<Sink, true, false, MODE>(p, grid, st);
    return count ? launch_t<Sink, false, true, MODE>(p, grid, st) : launch_t<Sink, false, false, MODE>(p, grid, st);
}

cudaError_t launch_sets(const SketchParams &p, int kind, bool bbit, bool count, int grid_fast, int grid_general,
                        cudaStream_t st) {
    // queue count and the two work counters are contiguous
    cudaError_t e = cudaMemsetAsync(p.queue_count, 0, 4 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (kind == kLsh) {
        if ((e = launch_mode<LshSink, 0>(p, false, count, grid_fast, st)) != cudaSuccess) return e;
        return launch_mode<LshSink, 1>(p, false, count, grid_general, st);
    }
    if (kind == kBottomK) {
        if ((e = launch_mode<BottomKSink, 0>(p, false, count, grid_fast, st)) != cudaSuccess) return e;
        return launch_mode<BottomKSink, 1>(p, false, count, grid_general, st);
    }
    if (p.key_row) {
        if ((e = launch_mode<RowSink, 0>(p, bbit, count, grid_fast, st)) != cudaSuccess) return e;
        return launch_mode<RowSink, 1>(p, bbit, count, grid_general, st);
    }
    if ((e = launch_mode<SketchSink, 0>(p, bbit, count, grid_fast, st)) != cudaSuccess) return e;
    return launch_mode<SketchSink, 1>(p, bbit, count, grid_general, st);
}

cudaError_t launch_batched(const SketchParams &p0, int kind, bool bbit, bool count, int grid_fast,
                           int grid_general, int grid_large, cudaStream_t st, const SideStream *side) {
    SketchParams p = p0;
    p.sched = 2;
    const bool lsh = kind != kSketch;           // bucket sinks: no block-per-set class
    if (lsh || grid_large <= 0) {
        p.large_nnz = 0;
        p.large_work = 0.f;
    }
    cudaError_t e = cudaMemsetAsync(p.queue_count, 0, kHeaderBytes, st);
    if (e != cudaSuccess) return e;
    const int cgrid = (int)((p.n_sets + 7) / 8 < 4096 ? (p.n_sets + 7) / 8 : 4096);
    classify_kernel<<<cgrid, 256, 0, st>>>(p);
    scan_kernel<<<1, 32, 0, st>>>(p);
    const int sgrid = (int)((p.n_sets + 255) / 256 < 4096 ? (p.n_sets + 255) / 256 : 4096);
    scatter_kernel<<<sgrid, 256, 0, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // With a side stream, the large sets' block kernel and then the general kernel over the sets
    // classified general run there, beside the fast kernel (none of them waits for another: each
    // takes the SMs the others leave, so the fast kernel's tail fills with general work); the
    // general kernel over the fast kernel's deferrals follows the fast kernel.  The fast kernel
    // is launched before the general one, so it is the first to fill the SMs.  Without one, the
    // large kernel runs first (its blocks become resident before the fast kernel's), then the
    // fast kernel, then the general kernel over every queued set.
    const bool large = !lsh && grid_large > 0 && (p.large_nnz > 0 || p.large_work > 0.f);
    if (side) {
        if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(side->st, side->fork, 0)) != cudaSuccess)
            return e;
    }
    cudaStream_t sst = side ? side->st : st;
    if (large) {
        if ((e = count ? (bbit ? launch_large<true, true>(p, grid_large, sst) : launch_large<false, true>(p, grid_large, sst))
                       : (bbit ? launch_large<true, false>(p, grid_large, sst) : launch_large<false, false>(p, grid_large, sst)))
            != cudaSuccess)
            return e;
    }
    SketchParams pa = p, pb = p;
    pa.gen_part = side ? 1 : 0;
    pb.gen_part = 2;
    auto run = [&](auto fast, auto general) -> cudaError_t {
        cudaError_t r;
        if ((r = fast(p, st)) != cudaSuccess) return r;
        if (side && (r = general(pa, sst)) != cudaSuccess) return r;
        return general(side ? pb : pa, st);
    };
    if (kind == kLsh)
        e = run([&](const SketchParams &q, cudaStream_t s) { return launch_mode<LshSink, 0>(q, false, count, grid_fast, s); },
                [&](const SketchParams &q, cudaStream_t s) { return launch_mode<LshSink, 1>(q, false, count, grid_general, s); });
    else if (kind == kBottomK)
        e = run([&](const SketchParams &q, cudaStream_t s) { return launch_mode<BottomKSink, 0>(q, false, count, grid_fast, s); },
                [&](const SketchParams &q, cudaStream_t s) { return launch_mode<BottomKSink, 1>(q, false, count, grid_general, s); });
    else if (p.key_row)
        e = run([&](const SketchParams &q, cudaStream_t s) { return launch_mode<RowSink, 0>(q, bbit, count, grid_fast, s); },
                [&](const SketchParams &q, cudaStream_t s) { return launch_mode<RowSink, 1>(q, bbit, count, grid_general, s); });
    else
        e = run([&](const SketchParams &q, cudaStream_t s) { return launch_mode<SketchSink, 0>(q, bbit, count, grid_fast, s); },
                [&](const SketchParams &q, cudaStream_t s) { return launch_mode<SketchSink, 1>(q, bbit, count, grid_general, s); });
    if (e != cudaSuccess) return e;
    if (side) {
        if ((e = cudaEventRecord(side->join, side->st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, side->join, 0)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

size_t sink_bytes(int kind, int k, int K, bool key_row) {
    return kind == kLsh ? lsh_sink_bytes(k, K)
                        : (kind == kBottomK ? bottomk_sink_bytes(k) : sketch_sink_bytes(k, key_row));
}

size_t warp_bytes(int kind, int k, int K, int mode, bool key_row) {
    const size_t sink = (sink_bytes(kind, k, K, key_row) + 15) & ~(size_t)15;
    return sink + (mode == 0 ? kFastPathBytes : kGenPathBytes);
}

// Shared memory limit of every kernel in this file.  The dynamic shared memory a launch may
// request above 48 KB is a per-function attribute of the device, so it is raised once per device,
// to the device's opt-in maximum, before the first launch (at context creation), and never
// changed afterwards: launches from several host threads with different shared-memory sizes then
// cannot race on it.  The attribute only bounds what a launch may request; each launch still
// gets exactly the bytes it asks for.
template <class Sink, bool BBIT, bool COUNT>
static cudaError_t allow_smem_sink(int bytes) {
    cudaError_t e = cudaFuncSetAttribute(set_kernel<Sink, BBIT, COUNT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(set_kernel<Sink, BBIT, COUNT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <class Sink>
static cudaError_t allow_smem_all(int bytes) {
    cudaError_t e = allow_smem_sink<Sink, false, false>(bytes);
    if (e == cudaSuccess) e = allow_smem_sink<Sink, false, true>(bytes);
    if (e == cudaSuccess) e = allow_smem_sink<Sink, true, false>(bytes);
    if (e == cudaSuccess) e = allow_smem_sink<Sink, true, true>(bytes);
    return e;
}

cudaError_t allow_max_shared_memory(int device) {
    static std::mutex mu;
    static bool done[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return cudaSuccess;
    int bytes = 0;
    cudaError_t e = cudaDeviceGetAttribute(&bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = allow_smem_all<SketchSink>(bytes);
    if (e == cudaSuccess) e = allow_smem_all<RowSink>(bytes);
    if (e == cudaSuccess) e = allow_smem_all<LshSink>(bytes);
    if (e == cudaSuccess) e = allow_smem_all<BottomKSink>(bytes);
    const void *large[8] = {(const void *)large_kernel<SketchSink, false, false>,
                            (const void *)large_kernel<SketchSink, false, true>,
                            (const void *)large_kernel<SketchSink, true, false>,
                            (const void *)large_kernel<SketchSink, true, true>,
                            (const void *)large_kernel<RowSink, false, false>,
                            (const void *)large_kernel<RowSink, false, true>,
                            (const void *)large_kernel<RowSink, true, false>,
                            (const void *)large_kernel<RowSink, true, true>};
    for (int i = 0; i < 8 && e == cudaSuccess; ++i)
        e = cudaFuncSetAttribute(large[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[device] = true;
    return e;
}

int blocks_per_sm(int kind, int mode, bool bbit, int warps_per_block, size_t smem, bool key_row) {
    const void *fn;
    if (kind == kLsh) fn = mode == 0 ? kernel_fn<LshSink, false, false, 0>() : kernel_fn<LshSink, false, false, 1>();
    else if (kind == kBottomK)
        fn = mode == 0 ? kernel_fn<BottomKSink, false, false, 0>() : kernel_fn<BottomKSink, false, false, 1>();
    else if (key_row) {
        if (mode == 0) fn = bbit ? kernel_fn<RowSink, true, false, 0>() : kernel_fn<RowSink, false, false, 0>();
        else fn = bbit ? kernel_fn<RowSink, true, false, 1>() : kernel_fn<RowSink, false, false, 1>();
    } else if (mode == 0) fn = bbit ? kernel_fn<SketchSink, true, false, 0>() : kernel_fn<SketchSink, false, false, 0>();
    else fn = bbit ? kernel_fn<SketchSink, true, false, 1>() : kernel_fn<SketchSink, false, false, 1>();
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * warps_per_block, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

}  // namespace dm
