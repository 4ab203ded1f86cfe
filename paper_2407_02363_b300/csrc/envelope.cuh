// Device code of passes Y and Z of the exact EDT (Sec. III-C, Alg. 1 Steps 2-4) for grids
// whose every dimension is at most 256; the stand-alone kernels are in envelope.cu, the
// persistent batch kernel in edt.cu.
//
// A tile is 32 columns of one line family over the whole line (pass Y: 32 adjacent columns
// (x, z) of slice z, along y; pass Z: a patch of 8 x 4 or 32 x 1 columns (x, y), along z),
// one lane per column, NB warps per tile (the m2 / m3 banding of Alg. 1): warp b owns band
// b, the positions [b * bl, (b + 1) * bl) of every line, bl = ceil(n / NB).  Global
// accesses are runs along x (32 columns in pass Y, 8 or 32 in pass Z).  The line tile is
// staged into shared memory by one TMA box load (no multicast).
//
//   build   every warp sweeps the valid positions of its band (rows / slices that hold a
//           site: the same for all 32 columns, so the sweep is warp-uniform) and keeps the
//           band's stack of proximate sites in place: entry t's input word moves to slot
//           lo + t of the tile (a slot the sweep has read already) and its position to the
//           byte array `pos`.  With h(p) = f(p) + p^2, site b (between a and c) is popped
//           when c overtakes b no later than b overtakes a:
//               (h_c - h_b)(b - a) <= (h_b - h_a)(c - b)            (ComputeProximateSite)
//   merge   warp 0 joins the bands' stacks of each column left to right (PBA's merge of the
//           band envelopes): the top T of the joined prefix is dropped while the entry S
//           below it and the next band's first entry F dominate it, and F while T and the
//           entry G above F dominate it.  Both stacks are lower convex hulls of the points
//           (2p, h_p), so this alternation stops at their bridge.  The kept range of every
//           band is published through shared memory.
//   query   every warp walks the joined envelope over its own band (QueryNearestSite):
//           it finds the entry nearest to the band's first voxel (the values at a fixed
//           voxel are unimodal along the envelope), then advances one voxel at a time;
//           the next entry q+1 is strictly nearer to voxel j than entry q iff
//               h_(q+1) - h_q < 2 j (p_(q+1) - p_q),
//           whose right side grows by a constant per voxel (ties keep the lower site).
//
// Pass Z's in-plane distance g = (x - x')^2 + (y - y')^2 of a packed site x' | y' << 8 is
// K + (x'^2 + y'^2) - 2 (x x' + y y') with K = x^2 + y^2: two byte dot products.
#pragma once
#include <climits>
#include <type_traits>

#include "vedt_internal.h"

namespace vedt {
namespace lenv {

constexpr int kC = 32;   // columns per tile (lanes)

__device__ __forceinline__ int find_tile_grid(const GridDesc *__restrict__ gd, int ng, int64_t t, bool z) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((z ? gd[mid].tz_begin : gd[mid].ty_begin) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Word-size policies of the two passes.  Grids with every dim <= 256 (small): 8-bit row
// sites, 16-bit 2-D sites x' | y' << 8, 8-bit stack positions, 32-bit products.  Grids
// with a dim above 256 (large, up to 1024): 16-bit row sites, 32-bit 2-D sites
// x' | y' << 16, 16-bit positions (pass Z keeps them in the free bits of its sites, so
// its tile needs no position array), 64-bit products in the domination test.  h(r, p) =
// f(p) + p^2 for input word r at position p stays below 2^22, and the walk's sums below
// 2^31, for lines up to 1024.  kCachedRepair: the merge keeps its four entries in
// registers (pass Z, where reloading an entry costs two dot products for h, or the
// unpacking of a packed position) or reloads them (pass Y, where h is two operations and
// the cache's bookkeeping costs as much as the reloads; both measured).

// Pass Y: input word = the row's nearest site x' (pass X); f(p) = (x - x')^2.
struct PolY {
    using In = uint8_t;
    using Pos = uint8_t;
    using Prod = int;
    using Out = uint16_t;   // the 2-D site x' | y' << 8
    static constexpr int kMax = 256, kOutShift = 8, kBig = 1 << 20;
    static constexpr bool kCachedRepair = false;
    static constexpr bool kPacked = false;
    int x;
    __device__ __forceinline__ int g(uint32_t r) const {
        const int d = x - static_cast<int>(r);
        return d * d;
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const { return g(r) + p * p; }
};

struct PolYL {
    using In = uint16_t;
    using Pos = uint16_t;
    using Prod = long long;
    using Out = uint32_t;   // x' | y' << 16
    static constexpr int kMax = 1024, kOutShift = 16, kBig = 1 << 23;
    static constexpr bool kCachedRepair = false;
    static constexpr bool kPacked = false;
    int x;
    __device__ __forceinline__ int g(uint32_t r) const {
        const int d = x - static_cast<int>(r);
        return d * d;
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const { return g(r) + p * p; }
};

// Pass Z: input word = the slice's nearest 2-D site x' | y' << 8 (pass Y);
// f(p) = (x - x')^2 + (y - y')^2 = K + dp(r, r) - 2 dp(r, x | y << 8).
struct PolZ {
    using In = uint16_t;
    using Pos = uint8_t;
    using Prod = int;
    static constexpr int kMax = 256, kBig = 1 << 20;
    static constexpr bool kCachedRepair = true;
    static constexpr bool kPacked = false;
    uint32_t xy8;
    int K;
    __device__ static PolZ at(int x, int y) {
        return PolZ{static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 8), x * x + y * y};
    }
    __device__ __forceinline__ int g(uint32_t r) const {
        return static_cast<int>(__dp4a(r, r, static_cast<unsigned>(K))) - 2 * static_cast<int>(__dp4a(r, xy8, 0u));
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const {
        return static_cast<int>(__dp4a(r, r, static_cast<unsigned>(K + p * p))) -
               2 * static_cast<int>(__dp4a(r, xy8, 0u));
    }
    // linear index x' + X y' + XY z' of the site as a 2-way dot product (coef = 1 | X << 16)
    static __device__ __forceinline__ uint32_t coef(int X) { return 1u | (static_cast<uint32_t>(X) << 16); }
    __device__ __forceinline__ int index(uint32_t r, int c, uint32_t coef, int XY) const {
        return static_cast<int>(__dp2a_lo(coef, r, static_cast<unsigned>(XY * c)));
    }
};

// Large pass Z: input word x' | y' << 16 (x', y' < 1024); a stack entry keeps its
// position (< 1024) in bits 10-15 and 26-29, which the site leaves free.
struct PolZL {
    using In = uint32_t;
    using Pos = uint16_t;
    using Prod = long long;
    static constexpr int kMax = 1024, kBig = 1 << 23;
    static constexpr bool kCachedRepair = true;
    static constexpr bool kPacked = true;
    int x, y;
    __device__ static PolZL at(int x, int y) { return PolZL{x, y}; }
    __device__ __forceinline__ int g(uint32_t r) const {
        const int dx = x - static_cast<int>(r & 0x3FFu), dy = y - static_cast<int>((r >> 16) & 0x3FFu);
        return dx * dx + dy * dy;
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const { return g(r) + p * p; }
    // linear index x' + X y' + XY z' of the site (coef = X)
    static __device__ __forceinline__ uint32_t coef(int X) { return static_cast<uint32_t>(X); }
    __device__ __forceinline__ int index(uint32_t r, int c, uint32_t coef, int XY) const {
        return static_cast<int>(r & 0x3FFu) + static_cast<int>(coef) * static_cast<int>((r >> 16) & 0x3FFu) + XY * c;
    }
    static __device__ __forceinline__ uint32_t pack(uint32_t r, int c) {
        return r | (static_cast<uint32_t>(c & 63) << 10) | (static_cast<uint32_t>(c >> 6) << 26);
    }
    static __device__ __forceinline__ int pos_of(uint32_t r) {
        return static_cast<int>(((r >> 10) & 63u) | ((r >> 26) << 6));
    }
};

// b (between a and c) is dropped: c overtakes b no later than b overtakes a.
template <class Prod>
__device__ __forceinline__ bool dominated(int ca, int ha, int cb, int hb, int cc, int hc) {
    return static_cast<Prod>(hc - hb) * (cb - ca) <= static_cast<Prod>(hb - ha) * (cc - cb);
}

template <int NB, int MAX = 256>
struct Geo {
    static constexpr int kWords = (MAX / NB + 31) / 32;   // valid-mask words per band
    static __host__ __device__ constexpr int len(int n) { return (n + NB - 1) / NB; }
};

// rows of the staged tile: whole TMA boxes of up to kBox positions
__host__ __device__ constexpr int staged_rows(int n) { return n <= kBox ? n : (n + kBox - 1) / kBox * kBox; }

// Shared memory of one tile of n positions: the staged line tile [rows][32], the stack
// positions [NB * bl][32] (none where the policy packs them into the sites) and the
// published kept ranges (j, then i + 1, NB x 32 each, bytes for small grids, 16-bit words
// above).  The TMA barrier lives in the first 8 bytes of the j ranges, which are written
// only after every thread has passed its wait and the barrier is invalidated.  A 256-long
// small pass-Z tile with four bands takes 24,832 bytes (nine CTAs per SM), a pass-Y tile
// 16,640 (thirteen).
template <int NB, class P>
struct Layout {
    using Rng = typename std::conditional<(P::kMax > 256), uint16_t, uint8_t>::type;
    int pos_off, rng_off, bar_off, bytes;
    __host__ __device__ Layout(int n) {
        const int in_b = staged_rows(n) * kC * static_cast<int>(sizeof(typename P::In));
        pos_off = (in_b + 15) & ~15;
        const int pos_b = P::kPacked ? 0 : Geo<NB>::len(n) * NB * kC * static_cast<int>(sizeof(typename P::Pos));
        rng_off = pos_off + ((pos_b + 15) & ~15);
        bar_off = rng_off;
        bytes = rng_off + 2 * NB * kC * static_cast<int>(sizeof(Rng));
    }
};

// valid-position bitmask of band [lo, hi) from per-position byte flags (warp-uniform)
template <int W>
__device__ __forceinline__ void band_mask(const uint8_t *__restrict__ flags, int lo, int hi, int lane,
                                          uint32_t (&vm)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int q = lo + 32 * w + lane;
        vm[w] = __ballot_sync(0xffffffffu, q < hi && flags[q] != 0);
    }
}

// Stack of proximate sites of one band over its valid positions lo + 32 w + (bit of
// vm[w]), ascending; entry t ends in slot lo + t (input word in col, position in cp).
//
// The two top entries a (below) and b stay in registers.  The band's first valid site is
// pushed before the sweep with a sentinel below it that nothing dominates against
// (position b - 1, h_b + kBig, kBig above every h: the right side of the test is then
// below -kBig, the left side above -kBig / 2), so the bottom entry is never popped,
// every later push shifts b into a, and the pop test needs no size check; a pop reloads a
// from the slot two below the top, clamped to the band's first slot, and takes the
// sentinel again when one entry is left.
template <int W, class P>
__device__ __forceinline__ int build(const P &pol, typename P::In *col, typename P::Pos *cp, int lo,
                                     const uint32_t (&vm)[W], int cap, int32_t *err) {
    constexpr int kBig = P::kBig;
    using In = typename P::In;
    using Pos = typename P::Pos;
    In *const in0 = col + lo * kC;   // the band's first slot
    Pos *const ps0 = cp + lo * kC;
    // the band's first valid site is pushed before the sweep, with the sentinel below it
    uint32_t v[W];
    int first = -1;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        v[w] = vm[w];
        if (first < 0 && v[w]) {   // warp-uniform
            first = lo + 32 * w + __ffs(v[w]) - 1;
            v[w] &= v[w] - 1u;
        }
    }
    if (first < 0) return 0;
    const uint32_t r0 = col[first * kC];
    int cb = first, hb = pol.h(r0, first);
    const int cs = cb - 1, hs = hb + kBig;   // the sentinel below the bottom entry
    int ca = cs, ha = hs, k = 1;
    if constexpr (P::kPacked) {
        in0[0] = static_cast<In>(P::pack(r0, first));
    } else {
        in0[0] = static_cast<In>(r0);
        ps0[0] = static_cast<Pos>(first);
    }
    auto step = [&](int c) {
        const uint32_t r = col[c * kC];
        const int hc = pol.h(r, c);
        while (dominated<typename P::Prod>(ca, ha, cb, hb, c, hc)) {
            --k;
            cb = ca;
            hb = ha;
            const int s = max(k - 2, 0) * kC;
            int c2, h2;
            if constexpr (P::kPacked) {
                const uint32_t w2 = in0[s];
                c2 = P::pos_of(w2);
                h2 = pol.h(w2, c2);
            } else {
                c2 = ps0[s];
                h2 = pol.h(in0[s], c2);
            }
            const bool real = k >= 2;
            ca = real ? c2 : cs;
            ha = real ? h2 : hs;
        }
        if (in_range(k, cap, err)) {   // debug builds: the stack never outgrows its band
            if constexpr (P::kPacked) {
                in0[k * kC] = static_cast<In>(P::pack(r, c));
            } else {
                in0[k * kC] = static_cast<In>(r);
                ps0[k * kC] = static_cast<Pos>(c);
            }
        }
        ca = cb;
        ha = hb;
        cb = c;
        hb = hc;
        ++k;
    };
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint32_t bits = v[w];
        const int base = lo + 32 * w;
        if (bits != 0u && bits + (bits & (0u - bits)) == 0u) {   // one run of valid positions up to bit 31
#pragma unroll 4
            for (int c = base + __ffs(bits) - 1; c < base + 32; ++c) step(c);
        } else {
            while (bits) {
                const int c = base + __ffs(bits) - 1;
                bits &= bits - 1u;
                step(c);
            }
        }
    }
    return k;
}

// a[b] for a band index known only at run time (selects, no local memory)
template <int NB>
__device__ __forceinline__ int pick(const int (&a)[NB], int b) {
    int v = a[0];
#pragma unroll
    for (int u = 1; u < NB; ++u)
        if (b == u) v = a[u];
    return v;
}

// The joined envelope of one column: band b keeps its stack entries j[b] .. i[b] (none if
// j[b] > i[b]); the envelope is their concatenation in band order.
template <int NB, class P>
struct Joined {
    const typename P::In *col;   // this column's slots (stride kC)
    const typename P::Pos *cp;   // their positions (unused where the policy packs them)
    int bl;
    int j[NB], i[NB];
    int32_t *err;
    __device__ __forceinline__ void at(int s, int &c, uint32_t &r) const {
        if (!in_range(s, NB * bl, err)) {
            c = 0;
            r = 0;
            return;
        }
        r = col[s * kC];
        if constexpr (P::kPacked) c = P::pos_of(r);
        else c = cp[s * kC];
    }
    __device__ __forceinline__ bool nonempty(int b) const { return pick<NB>(j, b) <= pick<NB>(i, b); }
    // largest non-empty band below b, or -1
    __device__ __forceinline__ int prev_band(int b) const {
        int s = -1;
#pragma unroll
        for (int u = 0; u < NB; ++u)
            if (u < b && j[u] <= i[u]) s = u;
        return s;
    }
    // smallest non-empty band above b, or -1
    __device__ __forceinline__ int next_band(int b) const {
        int s = -1;
#pragma unroll
        for (int u = NB - 1; u >= 0; --u)
            if (u > b && j[u] <= i[u]) s = u;
        return s;
    }
    // One junction of the merge: the joined prefix (top band tb, its kept entries jt .. ti)
    // against band b (first kept entry jb of 0 .. ib).  Every step reloads T (the prefix's
    // top), S (the entry below it) and F (band b's first kept entry), and G (the entry
    // above F) where needed.
    __device__ __forceinline__ void junction_reload(const P &pol, int b, int ib, int &tb, int &ti, int &jt, int &jb) {
        for (;;) {
            int sb = tb, si = ti - 1;   // entry below the top
            if (si < jt) {
                sb = prev_band(tb);
                si = sb >= 0 ? pick<NB>(i, sb) : 0;
            }
            int cT, cF;
            uint32_t rT, rF;
            at(tb * bl + ti, cT, rT);
            at(b * bl + jb, cF, rF);
            const int hT = pol.h(rT, cT), hF = pol.h(rF, cF);
            if (sb >= 0) {
                int cS;
                uint32_t rS;
                at(sb * bl + si, cS, rS);
                if (dominated<typename P::Prod>(cS, pol.h(rS, cS), cT, hT, cF, hF)) {
                    if (--ti < jt) {   // the top band is used up: the band below takes over
#pragma unroll
                        for (int u = 0; u < NB; ++u)
                            if (u == tb) i[u] = ti;
                        tb = sb;
                        ti = si;
                        jt = pick<NB>(j, tb);
                    }
                    continue;
                }
            }
            if (jb < ib) {
                int cG;
                uint32_t rG;
                at(b * bl + jb + 1, cG, rG);
                if (dominated<typename P::Prod>(cT, hT, cF, hF, cG, pol.h(rG, cG))) {
                    ++jb;
                    continue;
                }
            }
            break;
        }
    }
    // The same junction with T, S, F and G kept in registers: dropping T makes S the top
    // and loads the next S, dropping F makes G the first entry and loads the next G, so a
    // step loads one entry instead of three or four.
    __device__ __forceinline__ void junction_cached(const P &pol, int b, int ib, int &tb, int &ti, int &jt, int &jb) {
        int cT, cF, cS = 0, hS = 0, cG = 0, hG = 0;
        uint32_t rT, rF;
        at(tb * bl + ti, cT, rT);
        at(b * bl + jb, cF, rF);
        int hT = pol.h(rT, cT), hF = pol.h(rF, cF);
        int sb, si;   // S's band (-1: no entry below T) and slot
        auto below = [&]() {
            sb = tb;
            si = ti - 1;
            if (si < jt) {
                sb = prev_band(tb);
                si = sb >= 0 ? pick<NB>(i, sb) : 0;
            }
            if (sb >= 0) {
                uint32_t rS;
                at(sb * bl + si, cS, rS);
                hS = pol.h(rS, cS);
            }
        };
        below();
        bool g_ok = false;   // G loaded for the current F
        for (;;) {
            if (sb >= 0 && dominated<typename P::Prod>(cS, hS, cT, hT, cF, hF)) {
                if (--ti < jt) {   // the top band is used up: the band below takes over
#pragma unroll
                    for (int u = 0; u < NB; ++u)
                        if (u == tb) i[u] = ti;
                    tb = sb;
                    ti = si;
                    jt = pick<NB>(j, tb);
                }
                cT = cS;
                hT = hS;
                below();
                continue;
            }
            if (jb < ib) {
                if (!g_ok) {
                    uint32_t rG;
                    at(b * bl + jb + 1, cG, rG);
                    hG = pol.h(rG, cG);
                    g_ok = true;
                }
                if (dominated<typename P::Prod>(cT, hT, cF, hF, cG, hG)) {
                    ++jb;
                    cF = cG;
                    hF = hG;
                    g_ok = false;
                    continue;
                }
            }
            break;
        }
    }
    // PBA-style merge of the band stacks of sizes k[b] (see the file comment)
    __device__ __forceinline__ void merge(const P &pol, const int (&k)[NB]) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            j[b] = 0;
            i[b] = k[b] - 1;
        }
        int tb = -1;   // top band of the joined prefix
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (k[b] == 0) continue;
            if (tb >= 0) {
                int jb = 0;
                // the top band's kept range in scalars; the arrays are written back only
                // when the top moves to another band and at the end of the junction
                int ti = pick<NB>(i, tb), jt = pick<NB>(j, tb);
                if constexpr (P::kCachedRepair) junction_cached(pol, b, k[b] - 1, tb, ti, jt, jb);
                else junction_reload(pol, b, k[b] - 1, tb, ti, jt, jb);
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    if (u == tb) i[u] = ti;
                    if (u == b) j[u] = jb;
                }
            }
            tb = b;
        }
    }
    // The entry of the joined envelope nearest to voxel lo, starting from band `band`'s
    // first kept entry (or the next non-empty band's, else the last entry): steps down
    // while the entry below is no farther.  Returns its slot and band; c, r, hq its
    // position, input word and h.
    __device__ __forceinline__ void start(const P &pol, int band, int lo, int &s, int &sb, int &c, uint32_t &r,
                                          int &hq) const {
        int b = nonempty(band) ? band : next_band(band);
        if (b < 0) {
            b = prev_band(band);
            s = b * bl + pick<NB>(i, b);
        } else {
            s = b * bl + pick<NB>(j, b);
        }
        at(s, c, r);
        hq = pol.h(r, c);
        for (;;) {
            int pb = b, ps = s - 1;
            if (ps < b * bl + pick<NB>(j, b)) {
                pb = prev_band(b);
                if (pb < 0) break;
                ps = pb * bl + pick<NB>(i, pb);
            }
            int c2;
            uint32_t r2;
            at(ps, c2, r2);
            const int h2 = pol.h(r2, c2);
            if (h2 - 2 * lo * c2 > hq - 2 * lo * c) break;
            b = pb;
            s = ps;
            c = c2;
            r = r2;
            hq = h2;
        }
        sb = b;
    }
    // next slot after s (in band sb) along the envelope; false at its end
    __device__ __forceinline__ bool next(int &s, int &sb, int &se) const {
        if (s < se) {
            ++s;
            return true;
        }
        const int nb = next_band(sb);
        if (nb < 0) return false;
        sb = nb;
        s = nb * bl + pick<NB>(j, nb);
        se = nb * bl + pick<NB>(i, nb);
        return true;
    }
};

// Line tile staging: TMA boxes of up to kBox positions x 32 columns (one box for lines
// up to 256; longer lines take whole boxes, the last one read past the line's end as
// zeros that no sweep visits).
template <class In>
__device__ __forceinline__ void load_tile(In *in, const CUtensorMap *map, int n, int x0, int c1, bool along_y,
                                          uint64_t *bar) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
    const int bb = n < kBox ? n : kBox;
    const int nbox = (n + bb - 1) / bb;
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(nbox * bb * kC * sizeof(In)));
    for (int b = 0; b < nbox; ++b) {
        In *dst = in + static_cast<size_t>(b) * bb * kC;
        if (along_y) tma_load_3d(dst, map, x0, b * bb, c1, bar);
        else tma_load_3d(dst, map, x0, c1, b * bb, bar);
    }
}

__device__ __forceinline__ void drain_after_timeout(uint64_t *bar, uint32_t phase) {
    for (uint32_t i = 0; i < (1u << 20); ++i)
        if (mbar_try_wait(bar, phase)) return;
}

// Builds the bands, merges (warp 0) and publishes the kept ranges of a staged tile.
// Returns false when no position of the line is valid (the same for every column).
// kOwnBar: the TMA barrier lives in the first bytes of the range area (stand-alone
// kernels, one tile per CTA) and is invalidated before the ranges overwrite it; else it
// is a separate barrier that the caller reuses with alternating phases.
template <int NB, bool kOwnBar, class P>
__device__ __forceinline__ bool envelope(const P &pol, typename P::In *in, typename P::Pos *pos, uint8_t *rng_bytes,
                                         const uint8_t *__restrict__ flags, int n, Joined<NB, P> &J, int &lo, int &hi,
                                         uint64_t *bar, uint32_t phase, int32_t *err, bool &ok) {
    using Rng = typename Layout<NB, P>::Rng;
    const int tid = threadIdx.x, lane = tid & 31, band = tid >> 5;
    const int bl = Geo<NB>::len(n);
    lo = band * bl;
    hi = min(n, lo + bl);
    uint32_t vm[Geo<NB, P::kMax>::kWords];
    band_mask(flags, lo, hi, lane, vm);
    ok = mbar_wait_bounded(bar, phase, err);
    if (!ok) {
        drain_after_timeout(bar, phase);
        (void)__syncthreads_or(0);
        return false;
    }
    const int k = build(pol, in + lane, pos + lane, lo, vm, bl, err);
    J.col = in + lane;
    J.cp = pos + lane;
    J.bl = bl;
    J.err = err;
    if constexpr (NB == 1) {
        J.j[0] = 0;
        J.i[0] = k - 1;
        return __syncthreads_or(k) != 0;
    } else {
        // first kept entry; stack size, then last kept + 1 (ri starts at byte 64 or later,
        // past the barrier)
        Rng *rj = reinterpret_cast<Rng *>(rng_bytes), *ri = rj + NB * kC;
        ri[tid] = static_cast<Rng>(k);
        if (!__syncthreads_or(k)) return false;
        if (band == 0) {
            if constexpr (kOwnBar) {
                if (tid == 0) mbar_inval(bar);   // every thread has passed its wait; rj overwrites it
                __syncwarp();
            }
            int kk[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) kk[b] = ri[b * kC + lane];
            J.merge(pol, kk);
            __syncwarp();   // every lane of warp 0 has read the sizes before they are overwritten
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                rj[b * kC + lane] = static_cast<Rng>(J.j[b]);
                ri[b * kC + lane] = static_cast<Rng>(J.i[b] + 1);
            }
        }
        __syncthreads();
        if (band != 0) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                J.j[b] = rj[b * kC + lane];
                J.i[b] = static_cast<int>(ri[b * kC + lane]) - 1;
            }
        }
        return true;
    }
}

// ------------------------------------------------------------------------------------
// pass Y: tile = (grid, slice z, columns x0 .. x0 + 31), line along y; writes the 2-D
// site x' | y' << 8 of every voxel and the slice's flag
// ------------------------------------------------------------------------------------
// One pass-Y tile (grid g, tile lt of that grid) with NB warps, staged into `smem` (layout
// Layout<NB, P>(Y)) through `bar` (current parity `phase`).  Returns false if the
// staging wait timed out (flagged in err).
template <int NB, bool kOwnBar, class P = PolY>
__device__ __forceinline__ bool tile_y(const GridDesc &G, const CUtensorMap *tmap, int lt, uint8_t *smem,
                                       uint64_t *bar, uint32_t phase, int32_t *err) {
    using Out = typename P::Out;
    const int tid = threadIdx.x, lane = tid & 31;
    const int Y = G.Y, Xp = G.Xp;
    const int tiles_x = Xp / kC;
    const int z = lt / tiles_x, x0 = (lt % tiles_x) * kC;
    const Layout<NB, P> L(Y);
    auto *in = reinterpret_cast<typename P::In *>(smem);
    auto *pos = reinterpret_cast<typename P::Pos *>(smem + L.pos_off);
    uint8_t *rng = smem + L.rng_off;
    if (tid == 0) load_tile(in, tmap, Y, x0, z, true, bar);
    const P pol{x0 + lane};
    Joined<NB, P> J;
    int lo, hi;
    bool ok;
    const bool any = envelope<NB, kOwnBar>(pol, in, pos, rng, G.row_has + static_cast<int64_t>(z) * Y, Y, J, lo, hi, bar,
                                                   phase, err, ok);
    if (!ok) return false;
    if (x0 == 0 && tid == 0) G.slice_has[z] = any ? 1 : 0;
    if (!any || lo >= hi) return true;   // an empty slice writes nothing: pass Z skips it
    int s, sb, c0;
    uint32_t r0;
    int h0;
    J.start(pol, tid >> 5, lo, s, sb, c0, r0, h0);
    int se = sb * J.bl + pick<NB>(J.i, sb);
    // next entry: dh = h1 - h0, dc2 = 2 (c1 - c0); no next entry: dh = INT_MAX
    int c1 = 0, h1 = 0, dh = INT_MAX, dc2 = 0;
    uint32_t r1 = 0;
    auto fetch = [&]() {
        if (J.next(s, sb, se)) {
            J.at(s, c1, r1);
            h1 = pol.h(r1, c1);
            dh = h1 - h0;
            dc2 = 2 * (c1 - c0);
        } else {
            dh = INT_MAX;
            dc2 = 0;
        }
    };
    fetch();
    int thr = lo * dc2;
    Out site = static_cast<Out>(r0 | (static_cast<uint32_t>(c0) << P::kOutShift));
    Out *out = static_cast<Out *>(G.s2);
    uint32_t off = static_cast<uint32_t>((z * Y + lo) * Xp + x0 + lane);
    const uint32_t lim = static_cast<uint32_t>(Xp * Y * G.Z);
    for (int jv = lo; jv < hi; ++jv) {
        if (dh < thr) {
            do {
                c0 = c1;
                r0 = r1;
                h0 = h1;
                fetch();
                thr = jv * dc2;
            } while (dh < thr);
            site = static_cast<Out>(r0 | (static_cast<uint32_t>(c0) << P::kOutShift));
        }
        if (in_range(off, lim, err)) out[off] = site;
        off += Xp;
        thr += dc2;
    }
    return true;
}

// ------------------------------------------------------------------------------------
// pass Z: tile = (grid, patch of PX x (32 / PX) columns (x, y) at (x0, y0)), line along z;
// writes sqdist and the nearest voxel's linear index
// ------------------------------------------------------------------------------------
// One pass-Z tile (grid g, tile lt of that grid), as tile_y (layout Layout<NB, P>(Z)).
// Lane l owns column (x0 + l % PX, y0 + l / PX); the TMA box (PX, 32 / PX, Z) lands as
// [z][lane] for either shape.  The valid positions (slices holding a site) are the same
// for every column, so the build stays warp-uniform; lanes past the grid's last row (a
// ragged last patch, read as zero words) compute but store nothing.
template <int NB, bool kOwnBar, int PX, class P = PolZ>
__device__ __forceinline__ bool tile_z(const GridDesc &G, const CUtensorMap *tmap, int lt, uint8_t *smem,
                                       uint64_t *bar, uint32_t phase, int32_t *err) {
    static_assert(PX == 8 || PX == 32, "pass-Z tiles are 8 x 4 or 32 x 1 columns");
    constexpr int PY = kC / PX;
    const int tid = threadIdx.x, lane = tid & 31;
    const int X = G.X, Y = G.Y, Z = G.Z, Xp = G.Xp;
    const int tiles_x = Xp / PX;
    const int y0 = (lt / tiles_x) * PY, x0 = (lt % tiles_x) * PX;
    const Layout<NB, P> L(Z);
    auto *in = reinterpret_cast<typename P::In *>(smem);
    auto *pos = reinterpret_cast<typename P::Pos *>(smem + L.pos_off);
    uint8_t *rng = smem + L.rng_off;
    if (tid == 0) load_tile(in, tmap, Z, x0, y0, false, bar);
    const int x = x0 + lane % PX, y = y0 + lane / PX;
    const P pol = P::at(x, y);
    Joined<NB, P> J;
    int lo, hi;
    bool ok;
    const bool any = envelope<NB, kOwnBar>(pol, in, pos, rng, G.slice_has, Z, J, lo, hi, bar, phase, err, ok);
    if (!ok) return false;
    const bool live = x < X && y < Y;
    const uint32_t plane = static_cast<uint32_t>(X * Y);
    uint32_t off = static_cast<uint32_t>(lo) * plane + static_cast<uint32_t>(live ? y * X + x : 0);
    const uint32_t lim = plane * static_cast<uint32_t>(Z);
    int32_t *sq = G.sqdist, *ix = G.idx;
    if (!any) {   // empty grid
        for (int jv = lo; jv < hi; ++jv) {
            if (live && in_range(off, lim, err)) {
                sq[off] = INT_MAX;
                ix[off] = -1;
            }
            off += plane;
        }
        return true;
    }
    if (lo >= hi) return true;
    const uint32_t coef = P::coef(X);
    const int XY = X * Y;
    int s, sb, c0;
    uint32_t r0;
    int h0;
    J.start(pol, tid >> 5, lo, s, sb, c0, r0, h0);
    int se = sb * J.bl + pick<NB>(J.i, sb);
    int c1 = 0, h1 = 0, dh = INT_MAX, dc2 = 0;
    uint32_t r1 = 0;
    auto fetch = [&]() {
        if (J.next(s, sb, se)) {
            J.at(s, c1, r1);
            h1 = pol.h(r1, c1);
            dh = h1 - h0;
            dc2 = 2 * (c1 - c0);
        } else {
            dh = INT_MAX;
            dc2 = 0;
        }
    };
    fetch();
    int thr = lo * dc2;
    // value at voxel jv of entry c0: v = g0 + (jv - c0)^2, kept incrementally
    int d = lo - c0;
    int v = h0 - c0 * c0 + d * d;
    int inc = 2 * d + 1;
    int id = pol.index(r0, c0, coef, XY);
    for (int jv = lo; jv < hi; ++jv) {
        if (dh < thr) {
            do {
                c0 = c1;
                r0 = r1;
                h0 = h1;
                fetch();
                thr = jv * dc2;
            } while (dh < thr);
            d = jv - c0;
            v = h0 - c0 * c0 + d * d;
            inc = 2 * d + 1;
            id = pol.index(r0, c0, coef, XY);
        }
        if (live && in_range(off, lim, err)) {
            sq[off] = v;
            ix[off] = id;
        }
        off += plane;
        v += inc;
        inc += 2;
        thr += dc2;
    }
    return true;
}

}  // namespace lenv
}  // namespace vedt
