// Exact 3-D Euclidean distance transform (Sec. III-C, Alg. 1) as three separable sweeps:
//
//   pass X  (Step 1, BandSweep + PropagateAcrossBand): for every voxel the nearest
//           occupied x in its row.  One warp per row, each lane owning a contiguous
//           segment of S voxels: the segment's occupancy becomes an S-bit mask, a warp
//           prefix-max / suffix-min of the segments' last / first occupied x carries the
//           sites across segments, and two register sweeps finish each segment.
//   pass Y  (Steps 2-3, ComputeProximateSite + QueryNearestSite in every slice): per
//           column (x, z) the lower envelope of the parabolas (x - x_s(y'))^2 + (y - y')^2.
//   pass Z  (Step 4, the same along the stacking axis): per column (x, y) the lower
//           envelope of g2(z') + (z - z')^2, producing sqdist and a nearest voxel index.
//
// Passes Y and Z run one 64-thread CTA per 32 adjacent columns: thread t owns column
// (t & 31), the lower warp the lower half of every line and the upper warp the upper half
// (the banding of Alg. 1 with m2 = m3 = 2), so every global access is coalesced across x
// and all lanes of a warp scan the same positions.  The tile (32 columns x the whole line)
// is staged into shared memory with TMA box loads.  Each thread keeps the stack of
// proximate sites of its half explicitly in shared memory; after a CTA barrier both
// threads of a column merge the two stacks at the junction, and each walks the merged
// envelope forward over its own half.  The domination test is exact integer arithmetic
// with h_s = f(s) + s^2:
//   b (above a) is dropped under c  iff  (h_c - h_b)(b - a) <= (h_b - h_a)(c - b),
// i.e. c overtakes b no later than b overtakes a.  In the query the next proximate site
// p+1 is strictly nearer to voxel j iff h_(p+1) - h_p < 2 j (c_(p+1) - c_p).
//
// Small mode (every dim <= 256): pass X writes 8-bit row sites plus a per-row flag,
// pass Y 16-bit packed 2-D sites (x | y << 8), stack entries are 8-bit.  Large mode (dims
// up to 1024): 16-bit row sites with an explicit "none", 32-bit packed sites
// (x | y << 16), 16-bit stack entries and 64-bit products in the domination test.
#include <climits>
#include <type_traits>

#include "vedt_internal.h"

namespace vedt {

// ------------------------------------------------------------------------------------
// pass X
// ------------------------------------------------------------------------------------
template <int S, bool SMALL>
__device__ __forceinline__ void pass_x_row(const GridDesc &G, int64_t lr, int lane) {
    constexpr int kNoLeft = -4096, kNoRight = 8192;
    const int x0 = S * lane;
    const int X = G.X, Xp = G.Xp;
    const uint8_t *row = G.occ + lr * X;
    uint32_t m = 0;
    if ((X & 3) == 0 && x0 + S <= X) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(row + x0);
#pragma unroll
        for (int q = 0; q < S / 4; ++q) {
            const uint32_t nz = __vcmpne4(__ldg(w + q), 0u) & 0x08040201u;
            m |= ((nz * 0x01010101u) >> 24) << (4 * q);
        }
    } else {
        for (int i = 0; i < S; ++i) {
            const int x = x0 + i;
            if (x < X && row[x]) m |= 1u << i;
        }
    }
    int lastp = m ? x0 + 31 - __clz(m) : kNoLeft;
    int firstp = m ? x0 + __ffs(m) - 1 : kNoRight;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, lastp, d);
        const int u = __shfl_down_sync(0xffffffffu, firstp, d);
        if (lane >= d) lastp = max(lastp, t);
        if (lane + d < 32) firstp = min(firstp, u);
    }
    const bool any = __shfl_sync(0xffffffffu, lastp, 31) >= 0;
    int L = __shfl_up_sync(0xffffffffu, lastp, 1);
    int R = __shfl_down_sync(0xffffffffu, firstp, 1);
    if (lane == 0) L = kNoLeft;
    if (lane == 31) R = kNoRight;
    int left[S], best[S];
    int cur = L;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        if ((m >> i) & 1u) cur = x0 + i;
        left[i] = cur;
    }
    cur = R;
#pragma unroll
    for (int i = S - 1; i >= 0; --i) {
        if ((m >> i) & 1u) cur = x0 + i;
        const int x = x0 + i;
        best[i] = (x - left[i] <= cur - x) ? left[i] : cur;
    }
    if (x0 < Xp) {
        if (SMALL) {
            uint32_t wv[S / 4];
#pragma unroll
            for (int q = 0; q < S / 4; ++q)
                wv[q] = (best[4 * q] & 0xFF) | ((best[4 * q + 1] & 0xFF) << 8) | ((best[4 * q + 2] & 0xFF) << 16) |
                        (static_cast<uint32_t>(best[4 * q + 3]) << 24);
            uint32_t *o = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(G.xs) + lr * Xp + x0);
#pragma unroll
            for (int q = 0; q < S / 4; q += 2) *reinterpret_cast<uint2 *>(o + q) = make_uint2(wv[q], wv[q + 1]);
            if (lane == 0) G.row_has[lr] = any ? 1 : 0;
        } else {
            uint32_t wv[S / 2];
#pragma unroll
            for (int q = 0; q < S / 2; ++q)
                wv[q] = any ? ((best[2 * q] & 0xFFFF) | (static_cast<uint32_t>(best[2 * q + 1]) << 16)) : 0xFFFFFFFFu;
            uint32_t *o = reinterpret_cast<uint32_t *>(static_cast<uint16_t *>(G.xs) + lr * Xp + x0);
#pragma unroll
            for (int q = 0; q < S / 2; q += 4)
                *reinterpret_cast<uint4 *>(o + q) = make_uint4(wv[q], wv[q + 1], wv[q + 2], wv[q + 3]);
        }
    }
}

template <int S, bool SMALL>
__global__ void __launch_bounds__(256) k_pass_x(const GridDesc *__restrict__ gd, int ng, int64_t rows_total) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int g = 0;
    for (int64_t r = warp; r < rows_total; r += nwarps) {
        while (g + 1 < ng && gd[g + 1].row_begin <= r) ++g;
        pass_x_row<S, SMALL>(gd[g], r - gd[g].row_begin, lane);
    }
}

// ------------------------------------------------------------------------------------
// common
// ------------------------------------------------------------------------------------
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
__device__ __forceinline__ void drain_after_timeout(uint64_t *bar, uint32_t phase) {
    for (uint32_t i = 0; i < (1u << 20); ++i)
        if (mbar_try_wait(bar, phase)) return;
}

constexpr int kCols = kEnvCols;   // columns per tile (one thread per column and half)
constexpr int kLanes = 2 * kTile;  // threads per pass-Y/Z CTA; stride of the stack arrays

template <bool SMALL>
struct Env {
    using Link = typename std::conditional<SMALL, uint8_t, uint16_t>::type;
    using XS = typename std::conditional<SMALL, uint8_t, uint16_t>::type;     // pass-X site
    using Site = typename std::conditional<SMALL, uint16_t, uint32_t>::type;  // pass-Y site
    using Prod = typename std::conditional<SMALL, int, long long>::type;
    static constexpr int kNoLink = SMALL ? 0xFF : 0xFFFF;
    static constexpr int kShift = SMALL ? 8 : 16;
    static constexpr uint32_t kMask = SMALL ? 0xFFu : 0xFFFFu;
};

// ------------------------------------------------------------------------------------
// Envelope along one line (Steps 2-3) in two bands: each thread builds the stack of
// proximate sites of its half of the line (stk[i * 64] = position of its i-th proximate
// site from the bottom), sweeping its positions upward and popping dominated sites.
//
// `Line` supplies for position q: raw(q) (input word), valid(q, raw) and
// h(raw, q^2) = f(q) + q^2.
// ------------------------------------------------------------------------------------
template <bool SMALL, class Line>
__device__ __forceinline__ int build_stack(int lo, int hi, typename Env<SMALL>::Link *stk, const Line &L) {
    using Prod = typename Env<SMALL>::Prod;
    int k = 0, a = 0, b = 0, ha = 0, hb = 0, dab = 0, wab = 0;
    int c2 = lo * lo;
    for (int c = lo; c < hi; c2 += 2 * c + 1, ++c) {
        const uint32_t r = L.raw(c);
        if (!L.valid(c, r)) continue;
        const int hc = L.h(r, c2);
        while (k >= 2 && static_cast<Prod>(hc - hb) * wab <= static_cast<Prod>(dab) * (c - b)) {
            --k;
            b = a;
            hb = ha;
            if (k >= 2) {
                a = stk[(k - 2) * kLanes];
                ha = L.h(L.raw(a), a * a);
                dab = hb - ha;
                wab = b - a;
            }
        }
        stk[k * kLanes] = static_cast<typename Env<SMALL>::Link>(c);
        dab = hc - hb;
        wab = c - b;
        a = b;
        ha = hb;
        b = c;
        hb = hc;
        ++k;
    }
    return k;
}

// Merged envelope of the two halves of a line: the lower half's stack kept up to entry
// i, then the upper half's stack from entry j on.  Only the junction can violate the
// envelope's ordering, so the top of the lower stack is dropped while the next site up
// dominates it, and the bottom of the upper stack while the site below does (both lanes
// of a line compute the same result independently).
template <bool SMALL, class Line>
struct Merged {
    const typename Env<SMALL>::Link *lo_stk, *up_stk;
    int i, j, kU, m;      // m = merged length
    __device__ __forceinline__ int at(int t) const {
        return t <= i ? lo_stk[t * kLanes] : up_stk[(t - i - 1 + j) * kLanes];
    }
    __device__ __forceinline__ void build(const Line &L, int kL) {
        using Prod = typename Env<SMALL>::Prod;
        i = kL - 1;
        j = 0;
        for (;;) {
            if (i >= 1 && j < kU) {
                const int a = lo_stk[(i - 1) * kLanes], b = lo_stk[i * kLanes], c = up_stk[j * kLanes];
                const int ha = L.h(L.raw(a), a * a), hb = L.h(L.raw(b), b * b), hc = L.h(L.raw(c), c * c);
                if (static_cast<Prod>(hc - hb) * (b - a) <= static_cast<Prod>(hb - ha) * (c - b)) {
                    --i;
                    continue;
                }
            }
            if (i >= 0 && j + 1 < kU) {
                const int a = lo_stk[i * kLanes], b = up_stk[j * kLanes], c = up_stk[(j + 1) * kLanes];
                const int ha = L.h(L.raw(a), a * a), hb = L.h(L.raw(b), b * b), hc = L.h(L.raw(c), c * c);
                if (static_cast<Prod>(hc - hb) * (b - a) <= static_cast<Prod>(hb - ha) * (c - b)) {
                    ++j;
                    continue;
                }
            }
            break;
        }
        m = (i + 1) + (kU - j);
    }
};

// Walks the merged envelope forward over voxels [lo, hi) and calls emit.site(c, raw)
// when the nearest proximate site changes and emit.put(val) per voxel, val = f(c) +
// (j - c)^2 kept incrementally.  The next site p+1 is nearer to voxel j iff
// h1 - h0 < 2 j (c1 - c0); that threshold is kept incrementally too.
template <bool SMALL, class Line, class Emit>
__device__ __forceinline__ void query_merged(const Merged<SMALL, Line> &M, int lo, int hi, bool upper,
                                             const Line &L, Emit &emit) {
    // starting entry: the bottom for the lower half; for the upper half the entry nearest
    // to voxel lo, searched from the junction
    int p = 0;
    if (upper) {
        p = M.i + 1 < M.m ? M.i + 1 : M.m - 1;
        int c = M.at(p);
        int v = L.h(L.raw(c), c * c) - 2 * lo * c;
        while (p > 0) {
            const int cb = M.at(p - 1);
            const int vb = L.h(L.raw(cb), cb * cb) - 2 * lo * cb;
            if (vb > v) break;
            --p;
            v = vb;
        }
    }
    int c0 = M.at(p);
    uint32_t r0 = L.raw(c0);
    int h0 = L.h(r0, c0 * c0);
    int c1 = 0, h1 = 0, dc2 = 0, dh = 0;
    uint32_t r1 = 0;
    const bool more0 = p + 1 < M.m;
    if (more0) {
        c1 = M.at(p + 1);
        r1 = L.raw(c1);
        h1 = L.h(r1, c1 * c1);
        dc2 = 2 * (c1 - c0);
        dh = h1 - h0;
    }
    bool more = more0;
    int thr = lo * dc2;          // 2 j (c1 - c0)
    int val = h0 - 2 * lo * c0 + lo * lo;
    int inc = 2 * (lo - c0) + 1; // val(j+1) - val(j)
    emit.site(c0, r0);
    for (int j = lo; j < hi; ++j) {
        if (more && dh < thr) {
            do {
                ++p;
                c0 = c1;
                r0 = r1;
                h0 = h1;
                more = p + 1 < M.m;
                if (more) {
                    c1 = M.at(p + 1);
                    r1 = L.raw(c1);
                    h1 = L.h(r1, c1 * c1);
                    dc2 = 2 * (c1 - c0);
                    dh = h1 - h0;
                    thr = j * dc2;
                }
            } while (more && dh < thr);
            val = h0 - 2 * j * c0 + j * j;
            inc = 2 * (j - c0) + 1;
            emit.site(c0, r0);
        }
        emit.put(val);
        val += inc;
        inc += 2;
        thr += dc2;
    }
}

// Both halves of 32 lines: thread tid owns line (tid & 31), warp (tid >> 5) the half.
// The stacks are [entry][64 threads]; `ks` is 64 ints of shared scratch.
template <bool SMALL, class Line, class Emit>
__device__ __forceinline__ void envelope_two_warps(int n, int tid, typename Env<SMALL>::Link *stack, int *ks,
                                                   const Line &L, Emit &emit, int &k_total) {
    const bool upper = tid >= kTile;
    const int half = (n + 1) >> 1;
    const int lo = upper ? half : 0, hi = upper ? n : half;
    typename Env<SMALL>::Link *own = stack + tid;
    const int k = build_stack<SMALL>(lo, hi, own, L);
    ks[tid] = k;
    __syncthreads();
    const int k_oth = ks[tid ^ kTile];
    const int kL = upper ? k_oth : k, kU = upper ? k : k_oth;
    k_total = kL + kU;
    Merged<SMALL, Line> M;
    M.lo_stk = stack + (tid & (kTile - 1));
    M.up_stk = M.lo_stk + kTile;
    M.kU = kU;
    if (kL + kU == 0) {
        for (int j = lo; j < hi; ++j) emit.put(INT_MAX);
        return;
    }
    M.build(L, kL);
    query_merged<SMALL>(M, lo, hi, upper, L, emit);
}

// ------------------------------------------------------------------------------------
// pass Y: tile = (grid, slice z, 16 columns x0..x0+15), line along y
// ------------------------------------------------------------------------------------

template <bool SMALL>
struct LineY {
    const typename Env<SMALL>::XS *col;   // this thread's column of the staged tile (stride 32)
    const uint8_t *rh;                    // small mode: row flags of the slice
    int x;
    __device__ __forceinline__ uint32_t raw(int q) const { return col[q * kCols]; }
    __device__ __forceinline__ bool valid(int q, uint32_t r) const { return SMALL ? rh[q] != 0 : r != kNoX; }
    __device__ __forceinline__ int h(uint32_t r, int q2) const {
        const int d = x - static_cast<int>(r);
        return d * d + q2;
    }
};

template <bool SMALL>
struct EmitY {
    typename Env<SMALL>::Site *po;
    int Xp;
    typename Env<SMALL>::Site v;
    __device__ __forceinline__ void site(int c, uint32_t r) {
        v = static_cast<typename Env<SMALL>::Site>(r | (static_cast<uint32_t>(c) << Env<SMALL>::kShift));
    }
    __device__ __forceinline__ void put(int val) {
        *po = val == INT_MAX ? static_cast<typename Env<SMALL>::Site>(~0u) : v;
        po += Xp;
    }
};

// One pass-Y tile (grid g, tile lt of that grid).  `phase` is the parity of the tile
// barrier's current phase; the barrier must have been initialised.  Returns false if
// the staging wait timed out.  Ends with a CTA barrier so the caller may reuse smem.
template <bool SMALL>
__device__ __forceinline__ bool tile_y(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm, int g,
                                       int64_t lt, uint8_t *smem, uint64_t *bar, uint32_t phase, int32_t *err) {
    using E = Env<SMALL>;
    using Link = typename E::Link;
    using XS = typename E::XS;
    using Site = typename E::Site;
    const int tid = threadIdx.x;
    const int Y = gd[g].Y, Xp = gd[g].Xp;
    const int tiles_x = Xp / kCols;
    const int z = static_cast<int>(lt / tiles_x);
    const int x0 = static_cast<int>(lt % tiles_x) * kCols;
    const int by = min(Y, kBox);
    const int nbox = (Y + by - 1) / by;
    const int half = (Y + 1) >> 1;
    const size_t in_bytes = static_cast<size_t>(nbox) * by * kCols * sizeof(XS);
    XS *in = reinterpret_cast<XS *>(smem);                                    // [nbox*by][32]
    Link *stack = reinterpret_cast<Link *>(smem + in_bytes);                  // [half][64]
    int *ks = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(stack + static_cast<size_t>(half) * kLanes) + 15) &
                                      ~uintptr_t(15));                        // [64]
    uint8_t *rh = reinterpret_cast<uint8_t *>(ks + kLanes);                   // [Y]
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(in_bytes));
        for (int b = 0; b < nbox; ++b)
            tma_load_3d(in + static_cast<size_t>(b) * by * kCols, &tm[2 * g], x0, b * by, z, bar);
    }
    if (SMALL) {
        const uint8_t *src = gd[g].row_has + static_cast<int64_t>(z) * Y;
        for (int q = tid; q < Y; q += kLanes) rh[q] = src[q];
    }
    __syncthreads();
    if (!mbar_wait_bounded(bar, phase, err)) {
        drain_after_timeout(bar, phase);
        __syncthreads();
        return false;
    }
    const int ci = tid & (kCols - 1);
    const int lo = tid >= kTile ? half : 0;
    const LineY<SMALL> L{in + ci, rh, x0 + ci};
    EmitY<SMALL> emit{reinterpret_cast<Site *>(gd[g].s2) + (static_cast<int64_t>(z) * Y + lo) * Xp + x0 + ci, Xp, 0};
    int k_total;
    envelope_two_warps<SMALL>(Y, tid, stack, ks, L, emit, k_total);
    if (x0 == 0 && tid == 0) gd[g].slice_has[z] = k_total > 0 ? 1 : 0;
    __syncthreads();
    return true;
}

template <bool SMALL>
__global__ void __launch_bounds__(kLanes) k_pass_y(const GridDesc *__restrict__ gd,
                                                   const CUtensorMap *__restrict__ tm, int ng, int32_t *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 0);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    tile_y<SMALL>(gd, tm, g, t - gd[g].ty_begin, smem, &bar, 0, err);
}

// ------------------------------------------------------------------------------------
// pass Z: tile = (grid, row y, 16 columns x0..x0+15), line along z
// ------------------------------------------------------------------------------------
template <bool SMALL>
struct LineZ {
    const typename Env<SMALL>::Site *col;
    const uint8_t *has;
    int x, y;
    __device__ __forceinline__ uint32_t raw(int q) const { return col[q * kCols]; }
    __device__ __forceinline__ bool valid(int q, uint32_t) const { return has[q] != 0; }
    __device__ __forceinline__ int h(uint32_t r, int q2) const {
        const int dx = x - static_cast<int>(r & Env<SMALL>::kMask);
        const int dy = y - static_cast<int>(r >> Env<SMALL>::kShift);
        return dx * dx + dy * dy + q2;
    }
};

template <bool SMALL>
struct EmitZ {
    int32_t *osq, *oix;
    int64_t plane;
    int X, XY;
    int32_t id;
    bool live;
    __device__ __forceinline__ void site(int c, uint32_t r) {
        id = static_cast<int32_t>(r & Env<SMALL>::kMask) + X * static_cast<int32_t>(r >> Env<SMALL>::kShift) + XY * c;
    }
    __device__ __forceinline__ void put(int val) {
        if (live) {
            *osq = val;
            *oix = val == INT_MAX ? -1 : id;
        }
        osq += plane;
        oix += plane;
    }
};

template <bool SMALL>
__device__ __forceinline__ bool tile_z(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm, int g,
                                       int64_t lt, uint8_t *smem, uint64_t *bar, uint32_t phase, int32_t *err) {
    using E = Env<SMALL>;
    using Link = typename E::Link;
    using Site = typename E::Site;
    const int tid = threadIdx.x;
    const int X = gd[g].X, Y = gd[g].Y, Z = gd[g].Z, Xp = gd[g].Xp;
    const int tiles_x = Xp / kCols;
    const int y = static_cast<int>(lt / tiles_x);
    const int x0 = static_cast<int>(lt % tiles_x) * kCols;
    const int bz = min(Z, kBox);
    const int nbox = (Z + bz - 1) / bz;
    const int half = (Z + 1) >> 1;
    const size_t in_bytes = static_cast<size_t>(nbox) * bz * kCols * sizeof(Site);
    Site *in = reinterpret_cast<Site *>(smem);                                  // [nbox*bz][32]
    Link *stack = reinterpret_cast<Link *>(smem + in_bytes);                    // [half][64]
    int *ks = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(stack + static_cast<size_t>(half) * kLanes) + 15) &
                                      ~uintptr_t(15));                          // [64]
    uint8_t *has = reinterpret_cast<uint8_t *>(ks + kLanes);                    // [Z]
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(in_bytes));
        for (int b = 0; b < nbox; ++b)
            tma_load_3d(in + static_cast<size_t>(b) * bz * kCols, &tm[2 * g + 1], x0, y, b * bz, bar);
    }
    for (int q = tid; q < Z; q += kLanes) has[q] = gd[g].slice_has[q];
    __syncthreads();
    if (!mbar_wait_bounded(bar, phase, err)) {
        drain_after_timeout(bar, phase);
        __syncthreads();
        return false;
    }
    const int ci = tid & (kCols - 1);
    const int lo = tid >= kTile ? half : 0;
    const int x = x0 + ci;
    const LineZ<SMALL> L{in + ci, has, x, y};
    const int64_t plane = static_cast<int64_t>(X) * Y;
    const int xc = x < X ? x : X - 1;   // padding columns build but never store
    const int64_t off = static_cast<int64_t>(lo) * plane + static_cast<int64_t>(y) * X + xc;
    EmitZ<SMALL> emit{gd[g].sqdist + off, gd[g].idx + off, plane, X, X * Y, -1, x < X};
    int k_total;
    envelope_two_warps<SMALL>(Z, tid, stack, ks, L, emit, k_total);
    __syncthreads();
    return true;
}

template <bool SMALL>
__global__ void __launch_bounds__(kLanes) k_pass_z(const GridDesc *__restrict__ gd,
                                                   const CUtensorMap *__restrict__ tm, int ng, int32_t *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 1);
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    tile_z<SMALL>(gd, tm, g, t - gd[g].tz_begin, smem, &bar, 0, err);
}

// ------------------------------------------------------------------------------------
// persistent EDT over a whole table: one launch, work items dequeued in order
//   [0, nX)            pass-X items (rows_per_item rows of one grid)
//   [nX, nX + nY)      pass-Y tiles, each waiting for its grid's pass-X items
//   [nX + nY, total)   pass-Z tiles, each waiting for its grid's pass-Y tiles
// A tile only ever waits for items with smaller indices, which were dequeued earlier by
// running CTAs that never wait on later items, so the launch always drains.  Every
// wait is bounded; on expiry the error word is flagged and the tile is skipped.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_count(const unsigned *p, unsigned target, int32_t *err,
                                           uint32_t limit = 1u << 24) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (ld_acquire(p) >= target) return true;
        __nanosleep(64);
    }
    atomicOr(err, kErrTimeout);
    return false;
}

// Self-test of the bounded wait: waits for a counter that nothing increments.
__global__ void k_wait_selftest(const unsigned *counter, uint32_t limit, int32_t *err) {
    if (threadIdx.x == 0) wait_count(counter, 1u, err, limit);
}

cudaError_t launch_wait_selftest(const unsigned *counter, uint32_t limit, int32_t *err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(counter, limit, err);
    return cudaGetLastError();
}

template <int S, bool SMALL>
__global__ void __launch_bounds__(kLanes) k_edt_persistent(const GridDesc *__restrict__ gd,
                                                           const CUtensorMap *__restrict__ tm, int ng,
                                                           PersistCounters cnt, int rows_per_item, int32_t *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned item_s;
    __shared__ int ok_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned nX = cnt.n_x, nY = cnt.n_y, total = cnt.n_x + cnt.n_y + cnt.n_z;
    if (tid == 0) mbar_init(&bar, 1);
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) item_s = atomicAdd(cnt.next, 1u);
        __syncthreads();
        const unsigned it = item_s;
        __syncthreads();
        if (it >= total) break;
        if (it < nX) {
            // grid owning this pass-X item
            int lo = 0, hi = ng - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (static_cast<unsigned>(gd[mid].xi_begin) <= it) lo = mid;
                else hi = mid - 1;
            }
            const int g = lo;
            const int64_t rows = static_cast<int64_t>(gd[g].Y) * gd[g].Z;
            const int64_t r0 = static_cast<int64_t>(it - gd[g].xi_begin) * rows_per_item;
            const int64_t r1 = min(rows, r0 + rows_per_item);
            for (int64_t r = r0 + warp; r < r1; r += kLanes / 32) pass_x_row<S, SMALL>(gd[g], r, lane);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_x + g, 1u);
            }
        } else if (it < nX + nY) {
            const int64_t t = it - nX;
            const int g = find_grid(gd, ng, t, 0);
            if (tid == 0) {
                const unsigned need = static_cast<unsigned>((static_cast<int64_t>(gd[g].Y) * gd[g].Z + rows_per_item - 1) /
                                                            rows_per_item);
                ok_s = wait_count(cnt.done_x + g, need, err);
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncthreads();
            if (ok_s) {
                tile_y<SMALL>(gd, tm, g, t - gd[g].ty_begin, smem, &bar, phase, err);
                phase ^= 1u;
            }
            if (tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_y + g, 1u);
            }
        } else {
            const int64_t t = it - nX - nY;
            const int g = find_grid(gd, ng, t, 1);
            if (tid == 0) {
                const unsigned need = static_cast<unsigned>(static_cast<int64_t>(gd[g].Xp / kCols) * gd[g].Z);
                ok_s = wait_count(cnt.done_y + g, need, err);
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncthreads();
            if (ok_s) {
                tile_z<SMALL>(gd, tm, g, t - gd[g].tz_begin, smem, &bar, phase, err);
                phase ^= 1u;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static size_t smem_y(const GridTable &t) {
    const int by = t.maxY > kBox ? kBox : t.maxY;
    const size_t rows = static_cast<size_t>((t.maxY + by - 1) / by) * by;
    const size_t xs = t.large ? 2 : 1, link = t.large ? 2 : 1;
    return rows * kCols * xs + static_cast<size_t>((t.maxY + 1) / 2) * kLanes * link + 16 + kLanes * 4 + t.maxY;
}

static size_t smem_z(const GridTable &t) {
    const int bz = t.maxZ > kBox ? kBox : t.maxZ;
    const size_t rows = static_cast<size_t>((t.maxZ + bz - 1) / bz) * bz;
    const size_t site = t.large ? 4 : 2, link = t.large ? 2 : 1;
    return rows * kCols * site + static_cast<size_t>((t.maxZ + 1) / 2) * kLanes * link + 16 + kLanes * 4 + t.maxZ;
}

cudaError_t launch_pass_x(const GridTable &t, cudaStream_t s) {
    if (t.rows == 0) return cudaSuccess;
    const int64_t want = (t.rows + 7) / 8;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int blocks = static_cast<int>(want < cap ? want : cap);
    if (!t.large) {
        k_pass_x<8, true><<<blocks, 256, 0, s>>>(t.desc, t.n, t.rows);
    } else if (t.maxXp <= 256) {
        k_pass_x<8, false><<<blocks, 256, 0, s>>>(t.desc, t.n, t.rows);
    } else if (t.maxXp <= 512) {
        k_pass_x<16, false><<<blocks, 256, 0, s>>>(t.desc, t.n, t.rows);
    } else {
        k_pass_x<32, false><<<blocks, 256, 0, s>>>(t.desc, t.n, t.rows);
    }
    return cudaGetLastError();
}

template <bool SMALL>
static cudaError_t launch_y_impl(const GridTable &t, cudaStream_t s) {
    const size_t sm = smem_y(t);
    cudaError_t e = cudaFuncSetAttribute(k_pass_y<SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    k_pass_y<SMALL><<<static_cast<unsigned>(t.tiles_y), kLanes, sm, s>>>(t.desc, t.tmaps, t.n, t.err);
    return cudaGetLastError();
}

template <bool SMALL>
static cudaError_t launch_z_impl(const GridTable &t, cudaStream_t s) {
    const size_t sm = smem_z(t);
    cudaError_t e = cudaFuncSetAttribute(k_pass_z<SMALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    k_pass_z<SMALL><<<static_cast<unsigned>(t.tiles_z), kLanes, sm, s>>>(t.desc, t.tmaps, t.n, t.err);
    return cudaGetLastError();
}

template <int S, bool SMALL>
static cudaError_t launch_persistent_impl(const GridTable &t, const PersistCounters &c, int ctas_per_sm,
                                          int rows_per_item, cudaStream_t s) {
    const size_t sy = smem_y(t), sz = smem_z(t);
    const size_t sm = sy > sz ? sy : sz;
    auto k = k_edt_persistent<S, SMALL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kLanes, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    const int64_t total = static_cast<int64_t>(c.n_x) + c.n_y + c.n_z;
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    if (blocks > total) blocks = total;
    if (blocks < 1) return cudaSuccess;
    k<<<static_cast<unsigned>(blocks), kLanes, sm, s>>>(t.desc, t.tmaps, t.n, c, rows_per_item, t.err);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const GridTable &t, const PersistCounters &c, int ctas_per_sm, int rows_per_item,
                              cudaStream_t s) {
    if (!t.large) return launch_persistent_impl<8, true>(t, c, ctas_per_sm, rows_per_item, s);
    if (t.maxXp <= 256) return launch_persistent_impl<8, false>(t, c, ctas_per_sm, rows_per_item, s);
    if (t.maxXp <= 512) return launch_persistent_impl<16, false>(t, c, ctas_per_sm, rows_per_item, s);
    return launch_persistent_impl<32, false>(t, c, ctas_per_sm, rows_per_item, s);
}

cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s) {
    if (t.tiles_y == 0) return cudaSuccess;
    return t.large ? launch_y_impl<false>(t, s) : launch_y_impl<true>(t, s);
}

cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s) {
    if (t.tiles_z == 0) return cudaSuccess;
    return t.large ? launch_z_impl<false>(t, s) : launch_z_impl<true>(t, s);
}

}  // namespace vedt
