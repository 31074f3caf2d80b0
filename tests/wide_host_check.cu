// Host run of the wide-range kernel's per-lane arithmetic -- test infrastructure only.
//
// dm_wide.cu's geometry, rank-cut, code and walk helpers also compile for the host.  This file
// drives them the way one lane of wide_kernel does, sequentially over a set's elements (the
// warp's lanes only split the elements; the minimum per bucket does not depend on the order),
// so that their exact integer arithmetic is checked against the oracle without a GPU.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dm_wide.cu"

static int poisson_host(uint32_t u, const uint32_t *T) {
    int x = 0;
    for (int n = 0; n < 12; ++n) x += u >= T[n];
    return x;
}

extern "C" int wide_host_sketch(const int64_t *indptr, const uint64_t *idx, const double *w, int64_t n, int k,
                                uint32_t t, uint64_t seed, double phi0, const uint32_t *T, uint64_t *out,
                                int *status) {
    dm::WideParams wp{};
    wp.indptr = indptr;
    wp.indices = idx;
    wp.weights = w;
    wp.n_sets = n;
    wp.k = k;
    wp.t = t;
    wp.sigma = dm::mix64(seed ^ dm::kSeedSalt);
    wp.phi0 = phi0;
    for (int64_t set = 0; set < n; ++set) {
        const int64_t beg = indptr[set], end = indptr[set + 1];
        double l1 = 0, mx = 0;
        int bad = 0;
        for (int64_t i = beg; i < end; ++i) {
            const double x = w[i];
            if (!(x >= 0.0) || std::isinf(x)) bad |= 1;
            else if (x >= 0x1p960) bad |= 2;
            else {
                l1 += x;
                mx = std::max(mx, x);
            }
        }
        int err = (bad & 1) ? DM_EINVAL : ((bad & 2) ? DM_ERANGE : 0);
        if (!err && mx > 0 && mx < 0x1p-990) err = DM_ERANGE;
        std::vector<uint64_t> slots(k, ~0ull);
        if (!err && l1 > 0) {
            uint32_t c = (uint32_t)(bits_of(phi0 / l1) >> 32);
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
                for (int64_t q = beg; q < end && !err; ++q) {
                    WideWalk s;
                    s.p = q;
                    s.end = q + 1;                  // one element: the next one is 32 positions on
                    bool live = s.start(wp, cut, err);
                    while (live && !err) {
                        uint64_t cc = dm::mix64(s.ctr);
                        const uint32_t nx = (uint32_t)poisson_host((uint32_t)(cc >> 32), T);
                        uint32_t uthr = 1u << 24;
                        if (s.top) {
                            const uint64_t rb = s.r << 24;
                            uthr = s.Q <= rb ? 0u : (uint32_t)std::min(s.Q - rb, (uint64_t)(1u << 24));
                        }
                        const uint32_t vmax = (s.nu == s.nu_top && s.w + 1 == s.ncols) ? s.vtop : dm::kUMask;
                        for (uint32_t j = 0; j < nx; ++j) {
                            cc += dm::kGolden;
                            const uint64_t d = dm::mix64(cc);
                            const uint32_t u = (uint32_t)(d >> 40), v = (uint32_t)(d >> 16) & dm::kUMask;
                            if (u < uthr && v <= vmax) {
                                const uint32_t code = wide_code((s.r << 24) | u, s.rho, s.nu);
                                const uint64_t qq = dm::mix64(d ^ dm::kSlotSalt);
                                const uint32_t sl = (uint32_t)(((uint64_t)(uint32_t)(qq >> 32) * (uint64_t)k) >> 32);
                                slots[sl] = std::min(slots[sl], ((uint64_t)code << 32) | (uint32_t)qq);
                            }
                        }
                        live = s.advance(wp, cut, err);
                    }
                }
                if (err) break;
                if (std::find(slots.begin(), slots.end(), ~0ull) == slots.end()) break;
                const bool one = !cut.G.tiny && cut.G.ez < 0 && cut.G.ez > -64 && cut.G.Z == (1ull << -cut.G.ez);
                cut.rho_lo = one ? cut.rho_top + 1 : cut.rho_top;
                cut.Gp = one ? Dy64{0, 0, 0, false} : cut.G;
                c += 1u << 20;
            }
        }
        status[set] = err;
        for (int j = 0; j < k; ++j) out[set * k + j] = err ? ~0ull : slots[j];
    }
    return 0;
}
