// Exact 3-D Euclidean distance transform (Sec. III-C, Alg. 1) as three separable sweeps:
//
//   pass X  (Step 1, BandSweep + PropagateAcrossBand): for every voxel the nearest
//           occupied x in its row.  One warp per row; the row's occupancy becomes a
//           bitmask with warp ballots and the nearest set bit on either side comes from
//           count-leading-zeros plus a warp prefix-max / suffix-min over the words.
//   pass Y  (Steps 2-3, ComputeProximateSite + QueryNearestSite in every slice): per
//           column (x, z) the lower envelope of the parabolas (x - x_s(y'))^2 + (y - y')^2.
//   pass Z  (Step 4, the same along the stacking axis): per column (x, y) the lower
//           envelope of g2(z') + (z - z')^2, producing sqdist and a nearest voxel index.
//
// Passes Y and Z run one warp per 32 adjacent columns (one lane per column, so every
// global access is coalesced across x).  The warp's input tile (32 columns x the whole
// line) is staged into shared memory with one or more TMA box loads; the stack of
// proximate sites lives in shared memory as back-links (each pushed site records the
// site below it), so the query sweeps the line backwards from the top of the stack.
// The domination test is exact integer arithmetic:
//   b is dropped under c (a below b)  iff  (h_c - h_b)(b - a) <= (h_b - h_a)(c - b),
// with h_s = f(s) + s^2, i.e. c overtakes b no later than b overtakes a.
#include <climits>
#include <type_traits>

#include "vedt_internal.h"

namespace vedt {

// ------------------------------------------------------------------------------------
// pass X
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_pass_x(const GridDesc *__restrict__ gd, int ng,
                                                int64_t rows_total) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int g = 0;
    for (int64_t r = warp; r < rows_total; r += nwarps) {
        while (g + 1 < ng && gd[g + 1].row_begin <= r) ++g;
        const int X = gd[g].X, Xp = gd[g].Xp;
        const int64_t lr = r - gd[g].row_begin;
        const uint8_t *row = gd[g].occ + lr * X;
        uint16_t *out = gd[g].xs + lr * Xp;
        const int P = Xp >> 5;
        uint32_t mine = 0;   // lane k keeps the occupancy bitmask of word k (x in [32k, 32k+32))
        for (int k = 0; k < P; ++k) {
            const int x = (k << 5) + lane;
            const uint32_t b = (x < X) ? row[x] : 0u;
            const uint32_t m = __ballot_sync(0xffffffffu, b != 0u);
            if (lane == k) mine = m;
        }
        // last occupied x in words <= lane (prefix max), first occupied x in words >= lane
        int wl = mine ? (lane << 5) + 31 - __clz(mine) : -1;
        int wf = mine ? (lane << 5) + __ffs(mine) - 1 : INT_MAX;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wl, d);
            const int u = __shfl_down_sync(0xffffffffu, wf, d);
            if (lane >= d) wl = max(wl, t);
            if (lane + d < 32) wf = min(wf, u);
        }
        int lex = __shfl_up_sync(0xffffffffu, wl, 1);
        int rex = __shfl_down_sync(0xffffffffu, wf, 1);
        if (lane == 0) lex = -1;
        if (lane == 31) rex = INT_MAX;
        for (int k = 0; k < P; ++k) {
            const uint32_t m = __shfl_sync(0xffffffffu, mine, k);
            const int L = __shfl_sync(0xffffffffu, lex, k);
            const int R = __shfl_sync(0xffffffffu, rex, k);
            const uint32_t lo = m & ((2u << lane) - 1u);   // bits <= lane
            const uint32_t hi = m & (0xffffffffu << lane);  // bits >= lane
            const int left = lo ? (k << 5) + 31 - __clz(lo) : L;
            const int right = hi ? (k << 5) + __ffs(hi) - 1 : R;
            const int x = (k << 5) + lane;
            int best;
            if (left < 0) best = (right == INT_MAX) ? int(kNoX) : right;
            else if (right == INT_MAX) best = left;
            else best = (x - left <= right - x) ? left : right;
            out[x] = static_cast<uint16_t>(best);
        }
    }
}

// ------------------------------------------------------------------------------------
// lower envelope along one line, one lane per line
// ------------------------------------------------------------------------------------
template <bool LARGE>
struct EnvTraits {
    using Link = typename std::conditional<LARGE, uint16_t, uint8_t>::type;
    using Site = typename std::conditional<LARGE, uint32_t, uint16_t>::type;
    using Prod = typename std::conditional<LARGE, long long, int>::type;
    static constexpr int kNoLink = LARGE ? 0xFFFF : 0xFF;
    static constexpr int kShift = LARGE ? 16 : 8;
    static constexpr uint32_t kMask = LARGE ? 0xFFFFu : 0xFFu;
};

// Builds the stack of proximate sites over positions 0..n-1.  `hof(q, h)` returns
// false if position q has no site, else sets h = f(q) + q^2.  link is this lane's
// column of the back-link array (stride 32).  Returns the stack size; the top site
// and its h are left in top / htop.
template <bool LARGE, class HOf>
__device__ __forceinline__ int build_envelope(int n, typename EnvTraits<LARGE>::Link *link, HOf hof,
                                              int &top, int &htop) {
    using T = EnvTraits<LARGE>;
    using Prod = typename T::Prod;
    int k = 0, a = 0, b = 0, ha = 0, hb = 0;
    for (int c = 0; c < n; ++c) {
        int hc;
        if (!hof(c, hc)) continue;
        while (k >= 2) {
            const Prod lhs = static_cast<Prod>(hc - hb) * static_cast<Prod>(b - a);
            const Prod rhs = static_cast<Prod>(hb - ha) * static_cast<Prod>(c - b);
            if (lhs > rhs) break;
            --k;
            b = a;
            hb = ha;
            if (k >= 2) {
                a = link[b * kTile];
                hof(a, ha);
            }
        }
        link[c * kTile] = static_cast<typename T::Link>(k >= 1 ? b : T::kNoLink);
        if (k >= 1) {
            a = b;
            ha = hb;
        }
        b = c;
        hb = hc;
        ++k;
    }
    top = b;
    htop = hb;
    return k;
}

// Sweeps j = n-1 .. 0, moving down the stack while the site below is no farther, and
// calls emit(j, site, value) with value = f(site) + (j - site)^2.
template <bool LARGE, class HOf, class Emit>
__device__ __forceinline__ void query_envelope(int n, const typename EnvTraits<LARGE>::Link *link,
                                               HOf hof, int top, int htop, Emit emit) {
    using T = EnvTraits<LARGE>;
    int cur = top, hc = htop;
    int prv = link[cur * kTile];
    int hp = 0;
    if (prv != T::kNoLink) hof(prv, hp);
    for (int j = n - 1; j >= 0; --j) {
        while (prv != T::kNoLink && (hp - hc) <= 2 * j * (prv - cur)) {
            cur = prv;
            hc = hp;
            prv = link[cur * kTile];
            if (prv != T::kNoLink) hof(prv, hp);
        }
        emit(j, cur, hc - 2 * j * cur + j * j);
    }
}

__device__ __forceinline__ int find_grid(const GridDesc *__restrict__ gd, int ng, int64_t t, int which) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t beg = which == 0 ? gd[mid].ty_begin : gd[mid].tz_begin;
        if (beg <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// After a timed-out wait, give copies still in flight a bounded chance to land before
// the CTA releases its shared memory.
__device__ __forceinline__ void drain_after_timeout(uint64_t *bar) {
    for (uint32_t i = 0; i < (1u << 20); ++i)
        if (mbar_try_wait(bar, 0)) return;
}

// ------------------------------------------------------------------------------------
// pass Y: tile = (grid, slice z, 32 columns x0..x0+31), line along y
// ------------------------------------------------------------------------------------
template <bool LARGE>
__global__ void __launch_bounds__(32) k_pass_y(const GridDesc *__restrict__ gd,
                                               const CUtensorMap *__restrict__ tm, int ng, int32_t *err) {
    using T = EnvTraits<LARGE>;
    using Link = typename T::Link;
    using Site = typename T::Site;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int lane = threadIdx.x;
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 0);
    const int Y = gd[g].Y, Xp = gd[g].Xp;
    const int tiles_x = Xp >> 5;
    const int64_t lt = t - gd[g].ty_begin;
    const int z = static_cast<int>(lt / tiles_x);
    const int x0 = static_cast<int>(lt % tiles_x) << 5;
    const int by = min(Y, kBox);
    const int nbox = (Y + by - 1) / by;
    uint16_t *in = reinterpret_cast<uint16_t *>(smem);                       // [nbox*by][32]
    Link *link = reinterpret_cast<Link *>(smem + static_cast<size_t>(nbox) * by * kTile * 2);
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(link + static_cast<size_t>(Y) * kTile) + 15) & ~uintptr_t(15));
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(nbox) * by * kTile * 2);
        for (int b = 0; b < nbox; ++b) tma_load_3d(in + static_cast<size_t>(b) * by * kTile, &tm[2 * g], x0, b * by, z, bar);
    }
    __syncwarp();
    if (!mbar_wait_bounded(bar, 0, err)) {
        drain_after_timeout(bar);
        return;
    }
    const int x = x0 + lane;
    const uint16_t *col = in + lane;
    Link *lk = link + lane;
    auto hof = [&](int q, int &h) -> bool {
        const int s = col[q * kTile];
        if (s == kNoX) return false;
        const int d = x - s;
        h = d * d + q * q;
        return true;
    };
    int top, htop;
    const int k = build_envelope<LARGE>(Y, lk, hof, top, htop);
    Site *out = reinterpret_cast<Site *>(gd[g].s2) + static_cast<int64_t>(z) * Y * Xp + x;
    if (x0 == 0 && lane == 0) gd[g].slice_has[z] = k > 0 ? 1 : 0;
    if (k == 0) {
        for (int j = 0; j < Y; ++j) out[static_cast<int64_t>(j) * Xp] = static_cast<Site>(~Site(0));
        return;
    }
    int last = -1;
    uint32_t xs = 0;
    query_envelope<LARGE>(Y, lk, hof, top, htop, [&](int j, int site, int) {
        if (site != last) {
            last = site;
            xs = col[site * kTile];
        }
        out[static_cast<int64_t>(j) * Xp] = static_cast<Site>(xs | (static_cast<uint32_t>(site) << T::kShift));
    });
}

// ------------------------------------------------------------------------------------
// pass Z: tile = (grid, row y, 32 columns x0..x0+31), line along z
// ------------------------------------------------------------------------------------
template <bool LARGE>
__global__ void __launch_bounds__(32) k_pass_z(const GridDesc *__restrict__ gd,
                                               const CUtensorMap *__restrict__ tm, int ng, int32_t *err) {
    using T = EnvTraits<LARGE>;
    using Link = typename T::Link;
    using Site = typename T::Site;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int lane = threadIdx.x;
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 1);
    const int X = gd[g].X, Y = gd[g].Y, Z = gd[g].Z, Xp = gd[g].Xp;
    const int tiles_x = Xp >> 5;
    const int64_t lt = t - gd[g].tz_begin;
    const int y = static_cast<int>(lt / tiles_x);
    const int x0 = static_cast<int>(lt % tiles_x) << 5;
    const int bz = min(Z, kBox);
    const int nbox = (Z + bz - 1) / bz;
    Site *in = reinterpret_cast<Site *>(smem);                                 // [nbox*bz][32]
    Link *link = reinterpret_cast<Link *>(smem + static_cast<size_t>(nbox) * bz * kTile * sizeof(Site));
    uint8_t *has = reinterpret_cast<uint8_t *>(link + static_cast<size_t>(Z) * kTile);
    uint64_t *bar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(has + Z) + 15) & ~uintptr_t(15));
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(nbox) * bz * kTile * sizeof(Site));
        for (int b = 0; b < nbox; ++b)
            tma_load_3d(in + static_cast<size_t>(b) * bz * kTile, &tm[2 * g + 1], x0, y, b * bz, bar);
    }
    for (int q = lane; q < Z; q += kTile) has[q] = gd[g].slice_has[q];
    __syncwarp();
    if (!mbar_wait_bounded(bar, 0, err)) {
        drain_after_timeout(bar);
        return;
    }
    const int x = x0 + lane;
    const Site *col = in + lane;
    Link *lk = link + lane;
    auto hof = [&](int q, int &h) -> bool {
        if (!has[q]) return false;
        const uint32_t s = col[q * kTile];
        const int dx = x - static_cast<int>(s & T::kMask);
        const int dy = y - static_cast<int>(s >> T::kShift);
        h = dx * dx + dy * dy + q * q;
        return true;
    };
    int top, htop;
    const int k = build_envelope<LARGE>(Z, lk, hof, top, htop);
    if (x >= X) return;
    const int64_t plane = static_cast<int64_t>(X) * Y;
    int32_t *osq = gd[g].sqdist + static_cast<int64_t>(y) * X + x;
    int32_t *oix = gd[g].idx + static_cast<int64_t>(y) * X + x;
    if (k == 0) {
        for (int j = 0; j < Z; ++j) {
            osq[j * plane] = INT_MAX;
            oix[j * plane] = -1;
        }
        return;
    }
    int last = -1;
    int32_t id = 0;
    query_envelope<LARGE>(Z, lk, hof, top, htop, [&](int j, int site, int val) {
        if (site != last) {
            last = site;
            const uint32_t s = col[site * kTile];
            id = static_cast<int32_t>(s & T::kMask) +
                 X * (static_cast<int32_t>(s >> T::kShift) + Y * site);
        }
        osq[j * plane] = val;
        oix[j * plane] = id;
    });
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
static size_t smem_y(const GridTable &t) {
    const int by = t.maxY > kBox ? kBox : t.maxY;
    const size_t rows = static_cast<size_t>((t.maxY + by - 1) / by) * by;
    const size_t link = t.large ? 2 : 1;
    return rows * kTile * 2 + static_cast<size_t>(t.maxY) * kTile * link + 32;
}

static size_t smem_z(const GridTable &t) {
    const int bz = t.maxZ > kBox ? kBox : t.maxZ;
    const size_t rows = static_cast<size_t>((t.maxZ + bz - 1) / bz) * bz;
    const size_t site = t.large ? 4 : 2, link = t.large ? 2 : 1;
    return rows * kTile * site + static_cast<size_t>(t.maxZ) * kTile * link + t.maxZ + 32;
}

cudaError_t launch_pass_x(const GridTable &t, cudaStream_t s) {
    if (t.rows == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (t.rows + 7) / 8;
    const int blocks = static_cast<int>(want < sms * 16LL ? want : sms * 16LL);
    k_pass_x<<<blocks, 256, 0, s>>>(t.desc, t.n, t.rows);
    return cudaGetLastError();
}

template <bool LARGE>
static cudaError_t launch_y_impl(const GridTable &t, cudaStream_t s) {
    const size_t sm = smem_y(t);
    cudaError_t e = cudaFuncSetAttribute(k_pass_y<LARGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    k_pass_y<LARGE><<<static_cast<unsigned>(t.tiles_y), kTile, sm, s>>>(t.desc, t.tmaps, t.n, t.err);
    return cudaGetLastError();
}

template <bool LARGE>
static cudaError_t launch_z_impl(const GridTable &t, cudaStream_t s) {
    const size_t sm = smem_z(t);
    cudaError_t e = cudaFuncSetAttribute(k_pass_z<LARGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    k_pass_z<LARGE><<<static_cast<unsigned>(t.tiles_z), kTile, sm, s>>>(t.desc, t.tmaps, t.n, t.err);
    return cudaGetLastError();
}

cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s) {
    if (t.tiles_y == 0) return cudaSuccess;
    return t.large ? launch_y_impl<true>(t, s) : launch_y_impl<false>(t, s);
}

cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s) {
    if (t.tiles_z == 0) return cudaSuccess;
    return t.large ? launch_z_impl<true>(t, s) : launch_z_impl<false>(t, s);
}

}  // namespace vedt
