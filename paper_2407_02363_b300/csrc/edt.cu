// Exact 3-D Euclidean distance transform (Sec. III-C, Alg. 1) as three separable sweeps:
//
//   pass X  (Step 1, BandSweep + PropagateAcrossBand): for every voxel the nearest
//           occupied x in its row.  One warp per row, each lane owning a contiguous
//           segment of voxels: the segment's occupancy becomes a bit mask, a ballot of the
//           non-empty segments and two shuffles give each lane the nearest sites left and
//           right of its segment, and register sweeps finish each segment.
//   pass Y  (Steps 2-3, ComputeProximateSite + QueryNearestSite in every slice): per
//           column (x, z) the lower envelope of the parabolas (x - x_s(y'))^2 + (y - y')^2.
//   pass Z  (Step 4, the same along the stacking axis): per column (x, y) the lower
//           envelope of g2(z') + (z - z')^2, producing sqdist and a nearest voxel index.
//
// Passes Y and Z run one CTA of NB warps per tile of 32 columns (the m2 / m3 banding of
// Alg. 1): lane t owns column t, warp b the b-th band of every line, so all lanes of a
// warp scan the same positions.  The tile (32 columns x the whole line) is staged into
// shared memory with TMA box loads.  Each warp builds its band's stacks of proximate
// sites in place in the staged tile; after a CTA barrier warp 0 joins the bands of each
// column (the junction repair) and publishes the kept ranges, and every warp walks the
// merged envelope over its band.  The domination test is exact integer arithmetic with
// h_s = f(s) + s^2:
//   b (above a) is dropped under c  iff  (h_c - h_b)(b - a) <= (h_b - h_a)(c - b),
// i.e. c overtakes b no later than b overtakes a.  In the query the next proximate site
// p+1 is strictly nearer to voxel j iff h_(p+1) - h_p < 2 j (c_(p+1) - c_p).
//
// This file holds pass X for every size (k_pass_x_one and k_pass_x_small for grids with
// every dim <= 256: 8-bit row sites and a per-row flag; k_pass_x above: 16-bit row
// sites), passes Y and Z for grids above 256 (tile_y_small / tile_z_small with L = true:
// 16-bit row sites and stack positions, 32-bit packed 2-D sites x | y << 16, 64-bit
// products in the domination test; NB = 4 bands for lines up to 256, 8 beyond), and the
// two persistent batch kernels.  Passes Y and Z of grids with every dim <= 256 are in
// envelope.cu / envelope.cuh.
#include <climits>
#include <type_traits>

#include "envelope.cuh"
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
            if (lane == 0) G.row_has[lr] = any ? 1 : 0;
        }
    }
}

template <int S, bool SMALL>
__global__ void __launch_bounds__(256) k_pass_x(const GridDesc *__restrict__ gd, int ng, int64_t rows_total) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    int g = 0;
    for (int64_t r = warp; r < rows_total; r += nwarps) {
        while (g + 1 < ng && gd[g + 1].row_begin <= r) ++g;
        if (gd[g].changed && *gd[g].changed == 0) continue;   // unchanged since its last EDT
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
constexpr int kLanes = 2 * kTile;  // threads per CTA of the large-grid persistent kernel (two bands)

// ====================================================================================
// Pass X of grids with every dim <= 256: one warp per row, lane l owning voxels
// [8l, 8l + 8).  A ballot of the non-empty 8-byte segments ends an empty row (it only
// clears its flag: pass Y never reads its sites); otherwise the row's occupancy becomes
// one 8-bit mask per lane, and two shuffles give every lane the nearest occupied x left
// and right of its segment.  A segment with no site splits at the midpoint of those two;
// a segment with sites takes two register sweeps.
//
// Below it, the band tiles of passes Y and Z templated on the word sizes (L = true: grids
// above 256).  A band's stack of proximate sites lives in place: entry k keeps its staged
// input word in slot lo + k of the tile (a slot the sweep has already read) and its
// position in pos[k][tid], so a pop, the junction merge and the query read both words
// directly.
// ====================================================================================
__device__ __forceinline__ uint32_t nz_nibble(uint32_t w) {
    // bit i = (byte i != 0): set bit 7 of every non-zero byte, then gather bits 7, 15,
    // 23, 31 into bits 28..31 with one multiply (the partial products never overlap)
    const uint32_t t = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return (t * 0x00204081u) >> 28;
}

// occupancy bytes [x0, x0 + 8) of a row, zero beyond X
__device__ __forceinline__ uint2 row_bytes8(const uint8_t *row, int X, int x0, bool vec) {
    if (vec) return x0 < X ? __ldcs(reinterpret_cast<const uint2 *>(row + x0)) : make_uint2(0u, 0u);
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int x = x0 + i;
        const uint32_t b = x < X ? (row[x] != 0) : 0u;
        if (i < 4) lo |= b << (8 * i);
        else hi |= b << (8 * (i - 4));
    }
    return make_uint2(lo, hi);
}

// The same bytes after this frame's log-odds step (LogOdds): a voxel is a hit iff its
// occupancy byte is nonzero; the new log-odds and the 0/1 occupancy are stored back.
__device__ __forceinline__ uint2 row_logodds8(uint8_t *row, int8_t *lrow, int X, int x0, bool vec,
                                              const LogOdds &p) {
    if (vec) {
        if (x0 >= X) return make_uint2(0u, 0u);
        uint2 o = *reinterpret_cast<const uint2 *>(row + x0);
        uint2 l = *reinterpret_cast<const uint2 *>(lrow + x0);
        uint8_t *ob = reinterpret_cast<uint8_t *>(&o);
        int8_t *lb = reinterpret_cast<int8_t *>(&l);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int v = logodds_step(lb[b], ob[b] != 0, p);
            lb[b] = static_cast<int8_t>(v);
            ob[b] = v >= p.thr ? 1 : 0;
        }
        *reinterpret_cast<uint2 *>(row + x0) = o;
        *reinterpret_cast<uint2 *>(lrow + x0) = l;
        return o;
    }
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int x = x0 + i;
        if (x < X) {
            const int v = logodds_step(lrow[x], row[x] != 0, p);
            lrow[x] = static_cast<int8_t>(v);
            const uint32_t b = v >= p.thr ? 1u : 0u;
            row[x] = static_cast<uint8_t>(b);
            if (i < 4) lo |= b << (8 * i);
            else hi |= b << (8 * (i - 4));
        }
    }
    return make_uint2(lo, hi);
}

template <class I>   // row index type: int64_t for tables, int for one grid
__device__ __forceinline__ void pass_x_small_row(uint8_t *xs, uint8_t *row_has, int Xp, I lr, int lane, uint2 w) {
    constexpr int kNoLeft = -1024, kNoRight = 2048;
    // segments holding a site; an empty row (most rows of a sparse grid) stops here
    const uint32_t B = __ballot_sync(0xffffffffu, (w.x | w.y) != 0u);
    if (B == 0) {
        if (lane == 0) row_has[lr] = 0;
        return;
    }
    const uint32_t m = nz_nibble(w.x) | (nz_nibble(w.y) << 4);
    const int x0 = 8 * lane;
    const uint32_t below = B & ((1u << lane) - 1u);
    const uint32_t above = B & ~((2u << lane) - 1u);
    const int lastp = x0 + 31 - __clz(m);
    const int firstp = x0 + __ffs(m) - 1;
    int L = __shfl_sync(0xffffffffu, lastp, (31 - __clz(below)) & 31);
    int R = __shfl_sync(0xffffffffu, firstp, (__ffs(above) - 1) & 31);
    if (!below) L = kNoLeft;
    if (!above) R = kNoRight;
    uint32_t lo32, hi32;
    if (m == 0) {
        // voxels x <= floor((L + R) / 2) take L (ties go left), the rest R
        int nl = ((L + R) >> 1) - x0 + 1;
        nl = min(max(nl, 0), 8);
        const uint32_t rl = static_cast<uint32_t>(L & 0xFF) * 0x01010101u;
        const uint32_t rr = static_cast<uint32_t>(R & 0xFF) * 0x01010101u;
        const uint32_t ml = nl >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nl)) - 1u);
        const uint32_t mh = nl >= 8 ? 0xFFFFFFFFu : (nl <= 4 ? 0u : ((1u << (8 * (nl - 4))) - 1u));
        lo32 = (rl & ml) | (rr & ~ml);
        hi32 = (rl & mh) | (rr & ~mh);
    } else {
        int left[8], best[8];
        int cur = L;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((m >> i) & 1u) cur = x0 + i;
            left[i] = cur;
        }
        cur = R;
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            if ((m >> i) & 1u) cur = x0 + i;
            best[i] = (2 * (x0 + i) <= left[i] + cur) ? left[i] : cur;
        }
        lo32 = __byte_perm(__byte_perm(best[0], best[1], 0x0040), __byte_perm(best[2], best[3], 0x0040), 0x5410);
        hi32 = __byte_perm(__byte_perm(best[4], best[5], 0x0040), __byte_perm(best[6], best[7], 0x0040), 0x5410);
    }
    if (x0 < Xp) *reinterpret_cast<uint2 *>(xs + lr * Xp + x0) = make_uint2(lo32, hi32);
    if (lane == 0) row_has[lr] = 1;
}

// Grid-stride over rows in batches of kXRows rows per warp, the next batch's bytes
// loaded before the current batch is processed, so every warp keeps 2 * kXRows rows in
// flight.  The descriptor of the grid being swept stays in registers and is reloaded
// only when a row falls in another grid of the table.
constexpr int kXRows = 4;

template <bool INCR>
struct RowGrid {
    const uint8_t *occ;
    uint8_t *xs, *row_has;
    int64_t begin, end;
    int X, Xp;
    bool vec;
    bool skip = false;   // incremental map whose occupancy is unchanged since its last EDT
    int g = 0;
    // rows visited by one warp only increase, so the scan resumes from the current grid
    __device__ __forceinline__ void load(const GridDesc *__restrict__ gd, int ng, int64_t r) {
        while (g + 1 < ng && gd[g + 1].row_begin <= r) ++g;
        const GridDesc &G = gd[g];
        occ = G.occ;
        xs = static_cast<uint8_t *>(G.xs);
        row_has = G.row_has;
        begin = G.row_begin;
        end = G.row_begin + static_cast<int64_t>(G.Y) * G.Z;
        X = G.X;
        Xp = G.Xp;
        vec = (X & 7) == 0 && (reinterpret_cast<uintptr_t>(occ) & 7) == 0;
        if constexpr (INCR) skip = G.changed && *G.changed == 0;
    }
    __device__ __forceinline__ bool has(int64_t r) const { return r >= begin && r < end; }
};

// INCR: the table's grids may be incremental maps; rows of a grid whose occupancy is
// unchanged since its last EDT are skipped (the flag is read after the dependency wait).
// LO: the table is one grid with a log-odds occupancy `L`: each row's occupancy is
// updated (hits and misses of this frame, LogOdds p) as it is loaded.
template <bool INCR, bool LO>
__global__ void __launch_bounds__(256) k_pass_x_small(const GridDesc *__restrict__ gd, int ng, int64_t rows_total,
                                                      int8_t *__restrict__ L, LogOdds p) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t stride = nwarps * kXRows;
    int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    pdl_trigger();
    if (r >= rows_total) return;
    // one descriptor cache for the loads and one for the sweeps: each visits rows in
    // increasing order
    RowGrid<INCR> Gl, Gp;
    if constexpr (!INCR) {
        Gl.load(gd, ng, r);
        Gp.load(gd, ng, r);
    }
    pdl_wait();   // the occupancy (and the change flags) come from the previous kernels
    if constexpr (INCR) {
        Gl.load(gd, ng, r);
        Gp.load(gd, ng, r);
    }
    auto load = [&](int64_t rr) {
        if (rr >= rows_total) return make_uint2(0u, 0u);
        if (!Gl.has(rr)) Gl.load(gd, ng, rr);
        if (INCR && Gl.skip) return make_uint2(0u, 0u);
        if constexpr (LO)
            return row_logodds8(const_cast<uint8_t *>(Gl.occ) + (rr - Gl.begin) * Gl.X, L + (rr - Gl.begin) * Gl.X,
                                Gl.X, 8 * lane, Gl.vec, p);
        return row_bytes8(Gl.occ + (rr - Gl.begin) * Gl.X, Gl.X, 8 * lane, Gl.vec);
    };
    uint2 w[kXRows];
#pragma unroll
    for (int q = 0; q < kXRows; ++q) w[q] = load(r + q * nwarps);
    for (;;) {
        const int64_t rn = r + stride;
        uint2 wn[kXRows];
#pragma unroll
        for (int q = 0; q < kXRows; ++q) wn[q] = load(rn + q * nwarps);
#pragma unroll
        for (int q = 0; q < kXRows; ++q) {
            const int64_t rr = r + q * nwarps;
            if (rr < rows_total) {
                if (!Gp.has(rr)) Gp.load(gd, ng, rr);
                if (!(INCR && Gp.skip)) pass_x_small_row(Gp.xs, Gp.row_has, Gp.Xp, rr - Gp.begin, lane, w[q]);
            }
        }
        if (rn >= rows_total) break;
        r = rn;
#pragma unroll
        for (int q = 0; q < kXRows; ++q) w[q] = wn[q];
    }
}

// Pass X of a table with one grid and no per-row options (a frame's map, or one map's
// EDT): the same rows and sweeps as k_pass_x_small, with the grid's descriptor in
// registers and 32-bit row offsets (dims <= 256: at most 65,536 rows of 256 bytes), which
// removes the per-row table bookkeeping from the instruction stream.
__global__ void __launch_bounds__(256) k_pass_x_one(const GridDesc *__restrict__ gd, int rows) {
    const int lane = threadIdx.x & 31;
    const int nwarps = static_cast<int>((gridDim.x * blockDim.x) >> 5);
    int r = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    pdl_trigger();
    if (r >= rows) return;
    // the descriptor comes from the host, not from the previous kernels
    const uint8_t *occ = gd->occ;
    uint8_t *xs = static_cast<uint8_t *>(gd->xs);
    uint8_t *row_has = gd->row_has;
    const int X = gd->X, Xp = gd->Xp;
    const bool vec = (X & 7) == 0 && (reinterpret_cast<uintptr_t>(occ) & 7) == 0;
    pdl_wait();   // the occupancy comes from the previous kernels
    auto load = [&](int rr) {
        return rr < rows ? row_bytes8(occ + rr * X, X, 8 * lane, vec) : make_uint2(0u, 0u);
    };
    const int stride = nwarps * kXRows;
    uint2 w[kXRows];
#pragma unroll
    for (int q = 0; q < kXRows; ++q) w[q] = load(r + q * nwarps);
    for (;;) {
        const int rn = r + stride;
        uint2 wn[kXRows];
#pragma unroll
        for (int q = 0; q < kXRows; ++q) wn[q] = load(rn + q * nwarps);
#pragma unroll
        for (int q = 0; q < kXRows; ++q) {
            const int rr = r + q * nwarps;
            if (rr < rows) pass_x_small_row(xs, row_has, Xp, rr, lane, w[q]);
        }
        if (rn >= rows) break;
        r = rn;
#pragma unroll
        for (int q = 0; q < kXRows; ++q) w[q] = wn[q];
    }
}

// Policies of the two envelope passes, for grids with every dim <= 256 (L = false: 8-bit
// positions, 8-bit row sites, 16-bit 2-D sites x' | y' << 8, 32-bit products) and up to
// 1024 (L = true: 16-bit positions, 16-bit row sites, 32-bit 2-D sites x' | y' << 16,
// 64-bit products).  In = staged input word; h(raw, p) = f(p) + p^2 for that word at p.
template <bool L>
struct PolY {
    using In = typename std::conditional<L, uint16_t, uint8_t>::type;   // pass-X site x' of row p
    using Pos = typename std::conditional<L, uint16_t, uint8_t>::type;
    using Prod = typename std::conditional<L, long long, int>::type;
    static constexpr int kMax = L ? 1024 : 256;
    static constexpr bool kPacked = false;   // stack positions in a separate array
    int x;
    // squared distance within the line's plane, and with the position p along the line
    __device__ __forceinline__ int f(uint32_t r) const {
        const int d = x - static_cast<int>(r);
        return d * d;
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const { return f(r) + p * p; }
    static __device__ __forceinline__ uint32_t pack(uint32_t r, int) { return r; }
    static __device__ __forceinline__ int pos_of(uint32_t) { return 0; }
};

template <bool L>
struct PolZ {
    using In = typename std::conditional<L, uint32_t, uint16_t>::type;  // pass-Y 2-D site of slice p
    using Pos = typename std::conditional<L, uint16_t, uint8_t>::type;
    using Prod = typename std::conditional<L, long long, int>::type;
    static constexpr int kMax = L ? 1024 : 256;
    static constexpr int kShift = L ? 16 : 8;
    static constexpr uint32_t kMask = L ? 0x3FFu : 0xFFu;
    // Large mode keeps a stack entry's position (< 1024) in the bits its site leaves free
    // (10-15 and 26-29 of x' | y' << 16, x', y' < 1024), so the tile needs no position
    // array; small mode's 16-bit site has no free bits.
    static constexpr bool kPacked = L;
    int x, y;
    __device__ __forceinline__ int f(uint32_t r) const {
        const int dx = x - static_cast<int>(r & kMask), dy = y - static_cast<int>((r >> kShift) & kMask);
        return dx * dx + dy * dy;
    }
    __device__ __forceinline__ int h(uint32_t r, int p) const { return f(r) + p * p; }
    static __device__ __forceinline__ uint32_t pack(uint32_t r, int c) {
        return r | (static_cast<uint32_t>(c & 63) << 10) | (static_cast<uint32_t>(c >> 6) << 26);
    }
    static __device__ __forceinline__ int pos_of(uint32_t r) {
        return static_cast<int>(((r >> 10) & 63u) | ((r >> 26) << 6));
    }
};

// Banded line geometry of a tile: NB warps, warp b owns band [b * bl, min(n, (b + 1) * bl))
// of every line, bl = ceil(n / NB); lines are at most MAX long.
template <int NB, int MAX>
struct Bands {
    static constexpr int kWords = (MAX / NB + 31) / 32;   // valid-mask words per band
    static __host__ __device__ constexpr int len(int n) { return (n + NB - 1) / NB; }
};

// b dropped between a and c (positions a < b < c, h = f + p^2): c overtakes b no later
// than b overtakes a.  Products in Prod (64-bit once dims exceed 256).
template <class Prod>
__device__ __forceinline__ bool dominated(int ca, int ha, int cb, int hb, int cc, int hc) {
    return static_cast<Prod>(hc - hb) * (cb - ca) <= static_cast<Prod>(hb - ha) * (cc - cb);
}

// Stack of proximate sites of one band (Steps 2 and 4) over its valid positions
// lo + 32 w + (bit of vm[w]), ascending.  `col` = this column's input (stride kCols), the
// stack's input words are written back in place from slot lo; `cpos` = this column's
// positions (stride kTile), entry k's position kept in slot lo + k like its word.
template <int NB, class P>
__device__ __forceinline__ int small_build(const P &pol, typename P::In *col, typename P::Pos *cpos, int lo,
                                           const uint32_t (&vm)[Bands<NB, P::kMax>::kWords], int cap,
                                           int32_t *err) {
    using Prod = typename P::Prod;
    int k = 0, a = 0, b = 0, ha = 0, hb = 0, dab = 0, wab = 0;
    auto step = [&](int c) {
        if (!in_range(k, cap, err)) return;   // debug builds: the stack never outgrows its band
        const uint32_t r = col[c * kCols];
        const int hc = pol.h(r, c);
        while (k >= 2 && static_cast<Prod>(hc - hb) * wab <= static_cast<Prod>(dab) * (c - b)) {
            --k;
            b = a;
            hb = ha;
            if (k >= 2) {
                const uint32_t ra = col[(lo + k - 2) * kCols];
                if constexpr (P::kPacked) a = P::pos_of(ra);
                else a = cpos[(lo + k - 2) * kTile];
                ha = pol.h(ra, a);
                dab = hb - ha;
                wab = b - a;
            }
        }
        if constexpr (P::kPacked) {
            col[(lo + k) * kCols] = static_cast<typename P::In>(P::pack(r, c));
        } else {
            col[(lo + k) * kCols] = static_cast<typename P::In>(r);
            cpos[(lo + k) * kTile] = static_cast<typename P::Pos>(c);
        }
        dab = hc - hb;
        wab = c - b;
        a = b;
        ha = hb;
        b = c;
        hb = hc;
        ++k;
    };
#pragma unroll
    for (int w = 0; w < Bands<NB, P::kMax>::kWords; ++w) {
        uint32_t bits = vm[w];
        const int base = lo + 32 * w;
        if (bits == 0xFFFFFFFFu) {   // a run of 32 valid positions (warp-uniform)
#pragma unroll 2
            for (int c = base; c < base + 32; ++c) step(c);
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

// a[b] for a band index known only at run time (selects; no local memory)
template <int NB>
__device__ __forceinline__ int pick(const int (&a)[NB], int b) {
    int v = a[0];
#pragma unroll
    for (int u = 1; u < NB; ++u)
        if (b == u) v = a[u];
    return v;
}

// Merged envelope of a line's NB bands: band b keeps its stack entries j[b]..i[b] (none
// if j[b] > i[b]); the envelope is their concatenation in band order.
template <int NB, class P>
struct SmallMerged {
    typename P::In *in;         // this column's slots (stride kCols)
    const typename P::Pos *pos; // this column's positions, slot by slot (stride kTile)
    int bl;                     // band length
    int j[NB], i[NB];
    int last;                   // last non-empty band
    int32_t *err;               // error word (debug bounds checks)
    // entry of slot s = b * bl + t (band b's stack entry t)
    __device__ __forceinline__ void at_slot(int s, int &c, uint32_t &r) const {
        if (!in_range(s, NB * bl, err)) {
            c = 0;
            r = 0;
            return;
        }
        r = in[s * kCols];
        if constexpr (P::kPacked) c = P::pos_of(r);
        else c = pos[s * kTile];
    }
    __device__ __forceinline__ void at(int b, int t, int &c, uint32_t &r) const { at_slot(b * bl + t, c, r); }
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
    // Bands are joined left to right by the junction repair: the current top T is
    // popped while the entry S below it and the next band's first entry F dominate it,
    // and F is dropped while T and the entry G above F dominate it.  The four entries'
    // positions and h stay in registers, so each step loads one new entry.
    // entry below (sb, si + 1): (sb, si) itself if inside band sb's kept range, else the
    // top of the nearest earlier non-empty band; sb = -1 if there is none
    __device__ __forceinline__ void below(int &sb, int &si) const {
        if (si < pick<NB>(j, sb)) {
            sb = prev_band(sb);
            si = sb >= 0 ? pick<NB>(i, sb) : 0;
        }
    }
    __device__ __forceinline__ int hat(const P &pol, int b, int t, int &c) const {
        uint32_t r;
        at(b, t, c, r);
        return pol.h(r, c);
    }
    __device__ __forceinline__ void merge(const P &pol, const int (&k)[NB]) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            j[b] = 0;
            i[b] = k[b] - 1;
        }
        int tb = -1;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (k[b] == 0) continue;
            if (tb >= 0) {
                int jb = 0;
                const int ib = k[b] - 1;
                for (;;) {
                    const int ti = pick<NB>(i, tb), tj = pick<NB>(j, tb);
                    int sb = tb, si = ti - 1;
                    if (si < tj) {
                        sb = prev_band(tb);
                        si = sb >= 0 ? pick<NB>(i, sb) : 0;
                    }
                    int ca, cb, cc;
                    uint32_t ra, rb, rc;
                    at(tb, ti, cb, rb);
                    at(b, jb, cc, rc);
                    const int hb = pol.h(rb, cb), hc = pol.h(rc, cc);
                    if (sb >= 0) {
                        at(sb, si, ca, ra);
                        if (dominated<typename P::Prod>(ca, pol.h(ra, ca), cb, hb, cc, hc)) {
                            // pop the top; an emptied band hands the top to the band below
#pragma unroll
                            for (int u = 0; u < NB; ++u)
                                if (u == tb) i[u] = ti - 1;
                            if (ti - 1 < tj) tb = sb;
                            continue;
                        }
                    }
                    if (jb + 1 <= ib) {
                        at(b, jb + 1, ca, ra);
                        if (dominated<typename P::Prod>(cb, hb, cc, hc, ca, pol.h(ra, ca))) {
                            ++jb;
                            continue;
                        }
                    }
                    break;
                }
                j[b] = jb;
            }
            tb = b;   // a band's last entry can only be dropped by a later band
        }
        last = tb;
    }
    // last non-empty band from the ranges
    __device__ __forceinline__ void find_last() {
        last = -1;
#pragma unroll
        for (int u = 0; u < NB; ++u)
            if (j[u] <= i[u]) last = u;
    }
};

// Position of the walk's first entry: band b, stack entry t.
template <int NB, class P>
struct Cursor {
    int b, t;
    __device__ __forceinline__ void set(const SmallMerged<NB, P> &, int bb, int tt) {
        b = bb;
        t = tt;
    }
};

// Forward cursor of the walk over slots: the current band's kept range, then the later
// non-empty bands' ranges queued in order (first slot | last slot << 16), so a step
// needs no band search.
template <int NB, class P>
struct Walk {
    static constexpr int kQ = NB > 1 ? NB - 1 : 1;
    int s, se;
    uint32_t q[kQ];
    __device__ __forceinline__ void init(const SmallMerged<NB, P> &M, int b, int t) {
        s = b * M.bl + t;
        se = b * M.bl + pick<NB>(M.i, b);
#pragma unroll
        for (int k = 0; k < kQ; ++k) q[k] = ~0u;
        int n = 0;
#pragma unroll
        for (int u = 1; u < NB; ++u) {
            const bool take = u > b && M.j[u] <= M.i[u];
            const uint32_t v = static_cast<uint32_t>(u * M.bl + M.j[u]) | (static_cast<uint32_t>(u * M.bl + M.i[u]) << 16);
#pragma unroll
            for (int k = 0; k < kQ; ++k)
                if (take && k == n) q[k] = v;
            n += take ? 1 : 0;
        }
    }
    // next entry; false at the end of the envelope
    __device__ __forceinline__ bool next() {
        if (s < se) {
            ++s;
            return true;
        }
        if (q[0] == ~0u) return false;
        s = static_cast<int>(q[0] & 0xFFFFu);
        se = static_cast<int>(q[0] >> 16);
#pragma unroll
        for (int k = 0; k + 1 < kQ; ++k) q[k] = q[k + 1];
        q[kQ - 1] = ~0u;
        return true;
    }
};

// Walks the merged envelope over voxels [lo, hi) of band `band`: emit.start(c, raw)
// whenever the nearest proximate site changes (and at lo), emit.put(value) once per voxel.
// Entry q+1 is strictly nearer to voxel j iff h1 - h0 < 2 j (c1 - c0), ties keeping the
// lower site.  The walk starts at the band's first entry (or the next band's), steps down
// while the entry below is no worse at lo (the values at lo are unimodal along the
// envelope), then moves up as the voxels advance, one entry ahead.
template <int NB, class P, class E>
__device__ __forceinline__ void small_query(const P &pol, const SmallMerged<NB, P> &M, int lo, int hi, int band,
                                            E &emit) {
    if (lo >= hi) return;
    int cb = (M.j[0] <= M.i[0] && band == 0) ? 0 : -1;
    if (cb < 0) cb = (pick<NB>(M.j, band) <= pick<NB>(M.i, band)) ? band : M.next_band(band);
    Cursor<NB, P> cur;
    if (cb < 0) cur.set(M, M.last, pick<NB>(M.i, M.last));
    else cur.set(M, cb, pick<NB>(M.j, cb));
    int c0;
    uint32_t r0;
    M.at(cur.b, cur.t, c0, r0);
    int h0 = pol.h(r0, c0);
    for (;;) {
        int pb = cur.b, pt = cur.t - 1;
        if (pt < pick<NB>(M.j, cur.b)) {
            pb = M.prev_band(cur.b);
            if (pb < 0) break;
            pt = pick<NB>(M.i, pb);
        }
        int c;
        uint32_t r;
        M.at(pb, pt, c, r);
        const int hb = pol.h(r, c);
        if (hb - 2 * lo * c > h0 - 2 * lo * c0) break;
        cur.set(M, pb, pt);
        c0 = c;
        r0 = r;
        h0 = hb;
    }
    Walk<NB, P> nxt;
    nxt.init(M, cur.b, cur.t);
    if constexpr (E::kValues) {
        // Values at the current voxel j of the current entry (v0 = h0 - 2 j c0 + j^2, step
        // i0) and of the next one (v1, i1; 2^30 when there is none, above any value reached
        // here): the next entry is strictly nearer iff v1 < v0.  The emitter writes v0.
        constexpr int kNone = 1 << 30;
        int c1 = 0, v1 = kNone, i1 = 0;
        uint32_t r1 = 0;
        int v0 = h0 - 2 * lo * c0 + lo * lo, i0 = 2 * (lo - c0) + 1;
        auto fetch = [&](int j) {
            if (nxt.next()) {
                M.at_slot(nxt.s, c1, r1);
                const int d = j - c1;
                v1 = pol.f(r1) + d * d;
                i1 = 2 * d + 1;
            } else {
                v1 = kNone;
                i1 = 0;
            }
        };
        fetch(lo);
        emit.start(c0, r0);
        for (int j = lo; j < hi; ++j) {
            if (v1 < v0) {
                do {
                    c0 = c1;
                    r0 = r1;
                    v0 = v1;
                    i0 = i1;
                    fetch(j);
                } while (v1 < v0);
                emit.start(c0, r0);
            }
            emit.put(v0);
            v0 += i0;
            i0 += 2;
            v1 += i1;
            i1 += 2;
        }
    } else {
        // Only the nearest site is emitted: the next entry is strictly nearer to voxel j
        // iff h1 - h0 < 2 j (c1 - c0), the right side kept incrementally.
        int c1 = 0, h1 = 0, dc2 = 0, dh = INT_MAX;
        uint32_t r1 = 0;
        auto fetch = [&]() {
            if (nxt.next()) {
                M.at_slot(nxt.s, c1, r1);
                h1 = pol.h(r1, c1);
                dc2 = 2 * (c1 - c0);
                dh = h1 - h0;
            } else {
                dh = INT_MAX;
                dc2 = 0;
            }
        };
        fetch();
        int thr = lo * dc2;
        emit.start(c0, r0);
        for (int j = lo; j < hi; ++j) {
            if (dh < thr) {
                do {
                    c0 = c1;
                    r0 = r1;
                    h0 = h1;
                    fetch();
                    thr = j * dc2;
                } while (dh < thr);
                emit.start(c0, r0);
            }
            emit.put(0);
            thr += dc2;
        }
    }
}

__device__ __forceinline__ int align16(int n) { return (n + 15) & ~15; }

// valid-position bitmask of band [lo, hi) from per-position flags (warp-uniform)
template <int W>
__device__ __forceinline__ void band_mask(const uint8_t *flags, int lo, int hi, int lane, uint32_t (&vm)[W]) {
    uint8_t f[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int q = lo + 32 * w + lane;
        f[w] = q < hi ? flags[q] : 0;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) vm[w] = __ballot_sync(0xffffffffu, f[w] != 0);
}

template <bool L>
struct EmitYs {
    using Site = typename std::conditional<L, uint32_t, uint16_t>::type;
    static constexpr bool kValues = false;   // emits the 2-D site only
    Site *s2;
    uint32_t off, Xp;
    Site v;
    uint32_t lim;   // elements of s2 (debug bounds checks)
    int32_t *err;
    __device__ __forceinline__ void start(int c, uint32_t r) {
        v = static_cast<Site>(r | (static_cast<uint32_t>(c) << (L ? 16 : 8)));
    }
    __device__ __forceinline__ void put(int) {
        if (in_range(off, lim, err)) s2[off] = v;
        off += Xp;
    }
};

template <bool L>
struct EmitZs {
    static constexpr bool kValues = true;    // emits the squared distance too
    int32_t *sq, *ix;
    uint32_t off, plane;
    int X, XY;
    bool live;
    int id;
    uint32_t lim;   // voxels of the grid (debug bounds checks)
    int32_t *err;
    __device__ __forceinline__ void start(int c, uint32_t r) {
        id = static_cast<int>(r & PolZ<L>::kMask) + X * static_cast<int>((r >> PolZ<L>::kShift) & PolZ<L>::kMask) +
             XY * c;
    }
    __device__ __forceinline__ void put(int val) {
        if (live && in_range(off, lim, err)) {
            sq[off] = val;
            ix[off] = id;
        }
        off += plane;
    }
};

// Shared memory of an envelope tile over lines of n positions: the staged line tile
// (whole TMA boxes of up to kBox positions x 32 columns), the position stacks, the stack
// sizes and the published kept ranges.
template <int NB, class P>
__host__ __device__ constexpr int tile_in_bytes(int n) {
    return ((n + kBox - 1) / kBox) * (n < kBox ? n : kBox) * kCols * static_cast<int>(sizeof(typename P::In));
}
template <int NB, class P>
__host__ __device__ constexpr int tile_pos_bytes(int n) {
    if (P::kPacked) return 0;
    return Bands<NB, P::kMax>::len(n) * NB * kTile * static_cast<int>(sizeof(typename P::Pos));
}
// Stack sizes and kept ranges per (band, column): 8 bits while a band holds at most 255
// positions.
template <int NB, class P>
using RangeIdx = typename std::conditional<(P::kMax / NB <= 255), uint8_t, uint16_t>::type;
template <int NB, class P>
__host__ __device__ constexpr int small_region_off(int n) {
    return ((tile_in_bytes<NB, P>(n) + 15) & ~15) + ((tile_pos_bytes<NB, P>(n) + 15) & ~15);
}
// The range area (2 x NB x 32 indices, at least 64 bytes) also holds the standalone
// kernels' TMA barrier in its first 8 bytes until the tile is staged.  A 256-long pass-Z
// line tile then takes 24,832 bytes: nine CTAs per SM.
template <int NB, class P>
__host__ __device__ constexpr int small_smem(int n) {
    return small_region_off<NB, P>(n) + 2 * NB * kTile * static_cast<int>(sizeof(RangeIdx<NB, P>));
}

constexpr int kNBY = 4;   // default bands per line in the standalone passes, dims <= 256
constexpr int kNBL = 8;   // bands per line once some dim exceeds 256, lines over 256 long
constexpr int kNBLs = 4;  // bands per line once some dim exceeds 256, lines up to 256 long

// One envelope tile over the staged line tile `in` (n positions x 32 columns), after
// its TMA loads were issued: builds the bands, merges, walks.  `flags` = validity of each
// position; `emit` starts at the thread's first voxel; `region` = the range area.  With
// kOwnBar the TMA barrier `bar` lies in the range area's first bytes and is invalidated
// before the ranges overwrite it.  Returns 1 iff the line has a valid position (the same
// for every column), else 0.
template <int NB, class P, bool kOwnBar, class E>
__device__ __forceinline__ int small_envelope(typename P::In *in, typename P::Pos *pos, uint8_t *region,
                                              const uint8_t *flags, int n, const P &pol, E &emit, uint64_t *bar,
                                              uint32_t phase, int32_t *err, bool &ok) {
    using RIdx = RangeIdx<NB, P>;
    const int tid = threadIdx.x, lane = tid & (kTile - 1), band = tid >> 5;
    const int bl = Bands<NB, P::kMax>::len(n);
    const int lo = band * bl, hi = min(n, lo + bl);
    uint32_t vm[Bands<NB, P::kMax>::kWords];
    band_mask(flags, lo, hi, lane, vm);
    ok = mbar_wait_bounded(bar, phase, err);
    if (!ok) return 0;
    const int k = small_build<NB>(pol, in + lane, pos + lane, lo, vm, bl, err);
    // [NB][32] first kept entry per band, then [NB][32] stack sizes, overwritten by the
    // last kept entry + 1; the second half starts at byte 64 or later, past the barrier
    RIdx *rj = reinterpret_cast<RIdx *>(region);
    RIdx *ri = rj + NB * kTile;
    ri[tid] = static_cast<RIdx>(k);
    if (!__syncthreads_or(k)) return 0;   // no valid position: the same for every column
    SmallMerged<NB, P> M;
    M.in = in + lane;
    M.pos = pos + lane;
    M.bl = bl;
    M.err = err;
    if (band == 0) {   // one merge per column, published to the other bands
        if constexpr (kOwnBar) {
            if (tid == 0) mbar_inval(bar);   // every thread has passed its wait
            __syncwarp();
        }
        int kk[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) kk[b] = ri[b * kTile + lane];
        M.merge(pol, kk);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            rj[b * kTile + lane] = static_cast<RIdx>(M.j[b]);
            ri[b * kTile + lane] = static_cast<RIdx>(M.i[b] + 1);
        }
    }
    __syncthreads();
    if (band != 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            M.j[b] = rj[b * kTile + lane];
            M.i[b] = static_cast<int>(ri[b * kTile + lane]) - 1;
        }
        M.find_last();
    }
    small_query<NB>(pol, M, lo, hi, band, emit);
    return 1;
}

// Issues the TMA loads of a line tile: boxes of up to kBox positions along the line.
template <class In>
__device__ __forceinline__ void load_line_tile(In *in, const CUtensorMap *map, int n, int x0, int c1, bool along_y,
                                               uint64_t *bar) {
    const int bb = n < kBox ? n : kBox;
    const int nbox = (n + bb - 1) / bb;
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(nbox * bb * kCols * sizeof(In)));
    for (int b = 0; b < nbox; ++b) {
        if (along_y) tma_load_3d(in + static_cast<size_t>(b) * bb * kCols, map, x0, b * bb, c1, bar);
        else tma_load_3d(in + static_cast<size_t>(b) * bb * kCols, map, x0, c1, b * bb, bar);
    }
}

// One pass-Y tile (grid g, slice z, columns x0..x0+31) with NB * 32 threads.  Same
// contract as tile_y: `phase` is the barrier's current parity; ends with a CTA barrier
// so the caller may reuse shared memory.  kOwnBar: `bar` lies in the tile's range area.
template <int NB, bool L, bool kOwnBar>
__device__ __forceinline__ bool tile_y_small(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                             int g, int64_t lt, uint8_t *smem, uint64_t *bar, uint32_t phase,
                                             int32_t *err) {
    using P = PolY<L>;
    using In = typename P::In;
    const int tid = threadIdx.x, lane = tid & (kTile - 1);
    const int Y = gd[g].Y, Xp = gd[g].Xp;
    const int tiles_x = Xp / kCols;
    const int z = static_cast<int>(static_cast<uint32_t>(lt) / static_cast<uint32_t>(tiles_x));
    const int x0 = static_cast<int>(static_cast<uint32_t>(lt) % static_cast<uint32_t>(tiles_x)) * kCols;
    In *in = reinterpret_cast<In *>(smem);                                        // [Y][32]
    auto *pos = reinterpret_cast<typename P::Pos *>(smem + align16(tile_in_bytes<NB, P>(Y)));
    uint8_t *region = smem + small_region_off<NB, P>(Y);
    if (tid == 0) load_line_tile(in, &tm[2 * g], Y, x0, z, true, bar);
    const int lo = (tid >> 5) * Bands<NB, P::kMax>::len(Y);
    const P pol{x0 + lane};
    EmitYs<L> e{static_cast<typename EmitYs<L>::Site *>(gd[g].s2),
                static_cast<uint32_t>((static_cast<int64_t>(z) * Y + lo) * Xp + x0 + lane), static_cast<uint32_t>(Xp),
                0, static_cast<uint32_t>(Xp * Y * gd[g].Z), err};
    bool ok;
    const int total = small_envelope<NB, P, kOwnBar>(in, pos, region, gd[g].row_has + static_cast<int64_t>(z) * Y, Y,
                                                     pol, e, bar, phase, err, ok);
    if (!ok) {
        drain_after_timeout(bar, phase);
        (void)__syncthreads_or(0);   // pairs with the first barrier of the others
        return false;
    }
    // an empty slice (the same for every column) writes no sites: pass Z skips it
    if (x0 == 0 && tid == 0) gd[g].slice_has[z] = total > 0 ? 1 : 0;
    __syncthreads();
    return true;
}

// One pass-Z tile (grid g, row y, columns x0..x0+31) with NB * 32 threads.
template <int NB, bool L, bool kOwnBar, int PX>
__device__ __forceinline__ bool tile_z_small(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                             int g, int64_t lt, uint8_t *smem, uint64_t *bar, uint32_t phase,
                                             int32_t *err) {
    using P = PolZ<L>;
    using In = typename P::In;
    static_assert(PX == 8 || PX == kCols, "pass-Z tiles are 8 x 4 or 32 x 1 columns");
    constexpr int PY = kCols / PX;   // the tile is PX x PY columns (x, y); lane l owns (l % PX, l / PX)
    const int tid = threadIdx.x, lane = tid & (kTile - 1);
    const int X = gd[g].X, Y = gd[g].Y, Z = gd[g].Z, Xp = gd[g].Xp;
    const int tiles_x = Xp / PX;
    const int y0 = static_cast<int>(static_cast<uint32_t>(lt) / static_cast<uint32_t>(tiles_x)) * PY;
    const int x0 = static_cast<int>(static_cast<uint32_t>(lt) % static_cast<uint32_t>(tiles_x)) * PX;
    In *in = reinterpret_cast<In *>(smem);                                        // [Z][32]
    auto *pos = reinterpret_cast<typename P::Pos *>(smem + align16(tile_in_bytes<NB, P>(Z)));
    uint8_t *region = smem + small_region_off<NB, P>(Z);
    if (tid == 0) load_line_tile(in, &tm[2 * g + 1], Z, x0, y0, false, bar);
    const int bl = Bands<NB, P::kMax>::len(Z);
    const int lo = (tid >> 5) * bl, hi = min(Z, lo + bl);
    const int x = x0 + lane % PX, y = y0 + lane / PX;
    const bool live = x < X && y < Y;   // a ragged last patch reads zero words past row Y - 1
    const uint32_t plane = static_cast<uint32_t>(X * Y);
    const P pol{x, y};
    EmitZs<L> e{gd[g].sqdist, gd[g].idx,
                static_cast<uint32_t>(lo) * plane + static_cast<uint32_t>(live ? y * X + x : 0), plane, X, X * Y,
                live, 0, plane * static_cast<uint32_t>(Z), err};
    bool ok;
    const int total = small_envelope<NB, P, kOwnBar>(in, pos, region, gd[g].slice_has, Z, pol, e, bar, phase, err,
                                                     ok);
    if (!ok) {
        drain_after_timeout(bar, phase);
        (void)__syncthreads_or(0);   // pairs with the first barrier of the others
        return false;
    }
    if (total == 0) {   // empty grid
        for (int j = lo; j < hi; ++j) {
            if (live) {
                e.sq[e.off] = INT_MAX;
                e.ix[e.off] = -1;
            }
            e.off += plane;
        }
    }
    __syncthreads();
    return true;
}

template <int NB, bool L>
__global__ void __launch_bounds__(NB * kTile) k_pass_y_small(const GridDesc *__restrict__ gd,
                                                             const CUtensorMap *__restrict__ tm, int ng,
                                                             int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 0);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + small_region_off<NB, PolY<L>>(gd[g].Y));
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // the staged tile and the validity flags come from the previous pass
    if (gd[g].changed && *gd[g].changed == 0) return;   // unchanged since its last EDT
    tile_y_small<NB, L, true>(gd, tm, g, t - gd[g].ty_begin, smem, bar, 0, err);
}

template <int NB, bool L, int PX>
__global__ void __launch_bounds__(NB * kTile) k_pass_z_small(const GridDesc *__restrict__ gd,
                                                             const CUtensorMap *__restrict__ tm, int ng,
                                                             int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_grid(gd, ng, t, 1);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + small_region_off<NB, PolZ<L>>(gd[g].Z));
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // the staged tile and the validity flags come from the previous pass
    if (gd[g].changed && *gd[g].changed == 0) return;   // unchanged since its last EDT
    tile_z_small<NB, L, true, PX>(gd, tm, g, t - gd[g].tz_begin, smem, bar, 0, err);
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

// Persistent EDT for tables with a grid above 256: the large-grid pass X and two-band
// large-grid tiles (tile_y_small / tile_z_small with 16-bit row sites and positions,
// 32-bit 2-D sites, 32 x 1 pass-Z tiles).  The tile area of shared memory is reused from
// tile to tile: every thread fences its generic accesses of a tile against the async
// proxy before the CTA barrier that precedes the next tile's TMA load into the same bytes.
template <int S>
__global__ void __launch_bounds__(kLanes) k_edt_persistent(const GridDesc *__restrict__ gd,
                                                           const CUtensorMap *__restrict__ tm, int ng,
                                                           PersistCounters cnt, int rows_per_item, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
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
            for (int64_t r = r0 + warp; r < r1; r += kLanes / 32) pass_x_row<S, false>(gd[g], r, lane);
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_x + g, 1u);
            }
        } else {
            const bool is_y = it < nX + nY;
            const int64_t t = is_y ? it - nX : it - nX - nY;
            const int g = find_grid(gd, ng, t, is_y ? 0 : 1);
            if (tid == 0) {
                const unsigned need =
                    is_y ? static_cast<unsigned>((static_cast<int64_t>(gd[g].Y) * gd[g].Z + rows_per_item - 1) /
                                                 rows_per_item)
                         : static_cast<unsigned>(static_cast<int64_t>(gd[g].Xp / kCols) * gd[g].Z);
                ok_s = wait_count(is_y ? cnt.done_x + g : cnt.done_y + g, need, err);
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes -> TMA reads
            }
            __syncthreads();
            if (ok_s) {
                if (is_y) tile_y_small<2, true, false>(gd, tm, g, t - gd[g].ty_begin, smem, &bar, phase, err);
                else tile_z_small<2, true, false, kCols>(gd, tm, g, t - gd[g].tz_begin, smem, &bar, phase, err);
                phase ^= 1u;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (is_y && tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_y + g, 1u);
            }
        }
    }
}

// Persistent EDT for tables whose grids all have dims <= 256, on the stand-alone passes'
// NB-band tiles (envelope.cuh).  Same in-order queue and bounded waits as above.  The
// tile area of shared memory is reused from tile to tile: every thread fences its generic
// accesses of a tile against the async proxy before the CTA barrier that precedes the
// next tile's TMA load, which writes the same bytes.
template <int NB, int PX>
__global__ void __launch_bounds__(NB * 32) k_env_persistent(const GridDesc *__restrict__ gd,
                                                            const CUtensorMap *__restrict__ tm, int ng,
                                                            PersistCounters cnt, int rows_per_item, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
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
            int lo = 0, hi = ng - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (static_cast<unsigned>(gd[mid].xi_begin) <= it) lo = mid;
                else hi = mid - 1;
            }
            const GridDesc &G = gd[lo];
            const int64_t rows = static_cast<int64_t>(G.Y) * G.Z;
            const int64_t r0 = static_cast<int64_t>(it - G.xi_begin) * rows_per_item;
            const int64_t r1 = min(rows, r0 + rows_per_item);
            const bool vec = (G.X & 7) == 0 && (reinterpret_cast<uintptr_t>(G.occ) & 7) == 0;
            for (int64_t r = r0 + warp; r < r1; r += NB)
                pass_x_small_row(static_cast<uint8_t *>(G.xs), G.row_has, G.Xp, r, lane,
                                 row_bytes8(G.occ + r * G.X, G.X, 8 * lane, vec));
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_x + lo, 1u);
            }
        } else {
            const bool is_y = it < nX + nY;
            const int64_t t = is_y ? it - nX : it - nX - nY;
            const int g = find_grid(gd, ng, t, is_y ? 0 : 1);
            const GridDesc &G = gd[g];
            if (tid == 0) {
                const unsigned need =
                    is_y ? static_cast<unsigned>((static_cast<int64_t>(G.Y) * G.Z + rows_per_item - 1) / rows_per_item)
                         : static_cast<unsigned>(static_cast<int64_t>(G.Xp / kCols) * G.Z);
                ok_s = wait_count(is_y ? cnt.done_x + g : cnt.done_y + g, need, err);
                __threadfence();
                asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes -> TMA reads
            }
            __syncthreads();
            if (ok_s) {
                if (is_y) lenv::tile_y<NB, false>(G, &tm[2 * g], static_cast<int>(t - G.ty_begin), smem, &bar, phase, err);
                else lenv::tile_z<NB, false, PX>(G, &tm[2 * g + 1], static_cast<int>(t - G.tz_begin), smem, &bar, phase,
                                                 err);
                phase ^= 1u;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (is_y && tid == 0) {
                __threadfence();
                atomicAdd(cnt.done_y + g, 1u);
            }
        }
    }
}

template <int NB, int PX>
static cudaError_t launch_env_persistent(const GridTable &t, const PersistCounters &c, int ctas_per_sm,
                                         int rows_per_item, cudaStream_t s) {
    const size_t sy = static_cast<size_t>(lenv::Layout<NB, uint8_t>(t.maxY).bytes);
    const size_t sz = static_cast<size_t>(lenv::Layout<NB, uint16_t>(t.maxZ).bytes);
    const size_t sm = sy > sz ? sy : sz;
    cudaError_t e = ensure_dyn_smem<k_env_persistent<NB, PX>>(sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_env_persistent<NB, PX>, NB * 32, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    const int64_t total = static_cast<int64_t>(c.n_x) + c.n_y + c.n_z;
    int64_t blocks = static_cast<int64_t>(sm_count()) * per_sm;
    if (blocks > total) blocks = total;
    if (blocks < 1) return cudaSuccess;
    // a plain launch: the queue's first items read the occupancy the previous kernels wrote
    k_env_persistent<NB, PX><<<static_cast<unsigned>(blocks), NB * 32, sm, s>>>(t.desc, t.tmaps, t.n, c, rows_per_item,
                                                                           t.err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------

cudaError_t launch_pass_x(const GridTable &t, cudaStream_t s, int8_t *logodds, const int *lo_param) {
    if (t.rows == 0) return cudaSuccess;
    const int64_t want = (t.rows + 7) / 8;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int blocks = static_cast<int>(want < cap ? want : cap);
    if (!t.large) {
        // one resident wave of warps, each keeping two rows in flight
        static int per_sm = 0;
        if (per_sm == 0) {
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pass_x_small<false, false>, 256, 0) !=
                    cudaSuccess ||
                occ < 1)
                occ = 1;
            per_sm = occ;
        }
        const int64_t cap_small = static_cast<int64_t>(sm_count()) * per_sm;
        const int64_t want_small = (t.rows + 8 * kXRows - 1) / (8 * kXRows);
        const int nb = static_cast<int>(want_small < cap_small ? want_small : cap_small);
        const LogOdds p = lo_param ? LogOdds{lo_param[0], lo_param[1], lo_param[2], lo_param[3], lo_param[4]}
                                   : LogOdds{0, 0, 0, 0, 0};
        if (t.n == 1 && !t.incr && !logodds) {
            static int per_sm_one = 0;
            if (per_sm_one == 0) {
                int occ = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pass_x_one, 256, 0) != cudaSuccess ||
                    occ < 1)
                    occ = 1;
                per_sm_one = occ;
            }
            const int64_t cap_one = static_cast<int64_t>(sm_count()) * per_sm_one;
            const int nb1 = static_cast<int>(want_small < cap_one ? want_small : cap_one);
            return launch_pdl(k_pass_x_one, dim3(nb1), dim3(256), 0, s, t.desc, static_cast<int>(t.rows));
        }
        if (logodds) {
            if (t.n != 1 || t.incr) return cudaErrorInvalidValue;
            return launch_pdl(k_pass_x_small<false, true>, dim3(nb), dim3(256), 0, s, t.desc, t.n, t.rows, logodds, p);
        }
        if (t.incr)
            return launch_pdl(k_pass_x_small<true, false>, dim3(nb), dim3(256), 0, s, t.desc, t.n, t.rows,
                              static_cast<int8_t *>(nullptr), p);
        return launch_pdl(k_pass_x_small<false, false>, dim3(nb), dim3(256), 0, s, t.desc, t.n, t.rows,
                          static_cast<int8_t *>(nullptr), p);
    } else if (t.maxXp <= 256) {
        return launch_pdl(k_pass_x<8, false>, dim3(blocks), dim3(256), 0, s, t.desc, t.n, t.rows);
    } else if (t.maxXp <= 512) {
        return launch_pdl(k_pass_x<16, false>, dim3(blocks), dim3(256), 0, s, t.desc, t.n, t.rows);
    } else {
        return launch_pdl(k_pass_x<32, false>, dim3(blocks), dim3(256), 0, s, t.desc, t.n, t.rows);
    }
}

template <int S>
static cudaError_t launch_persistent_impl(const GridTable &t, const PersistCounters &c, int ctas_per_sm,
                                          int rows_per_item, cudaStream_t s) {
    const size_t sy = small_smem<2, PolY<true>>(t.maxY), sz = small_smem<2, PolZ<true>>(t.maxZ);
    const size_t sm = sy > sz ? sy : sz;
    auto k = k_edt_persistent<S>;
    cudaError_t e = ensure_dyn_smem<k_edt_persistent<S>>(sm);
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
    if (!t.large) {
        if (t.pzx != 8 && t.pzx != 32) return cudaErrorInvalidValue;
        const bool p8 = t.pzx == 8;
        switch (t.bands) {
            case 1: return p8 ? launch_env_persistent<1, 8>(t, c, ctas_per_sm, rows_per_item, s)
                              : launch_env_persistent<1, 32>(t, c, ctas_per_sm, rows_per_item, s);
            case 2: return p8 ? launch_env_persistent<2, 8>(t, c, ctas_per_sm, rows_per_item, s)
                              : launch_env_persistent<2, 32>(t, c, ctas_per_sm, rows_per_item, s);
            case 8: return p8 ? launch_env_persistent<8, 8>(t, c, ctas_per_sm, rows_per_item, s)
                              : launch_env_persistent<8, 32>(t, c, ctas_per_sm, rows_per_item, s);
            default: return p8 ? launch_env_persistent<4, 8>(t, c, ctas_per_sm, rows_per_item, s)
                               : launch_env_persistent<4, 32>(t, c, ctas_per_sm, rows_per_item, s);
        }
    }
    if (t.pzx != kCols) return cudaErrorInvalidValue;   // its pass-Z tiles are 32 x 1 rows
    if (t.maxXp <= 256) return launch_persistent_impl<8>(t, c, ctas_per_sm, rows_per_item, s);
    if (t.maxXp <= 512) return launch_persistent_impl<16>(t, c, ctas_per_sm, rows_per_item, s);
    return launch_persistent_impl<32>(t, c, ctas_per_sm, rows_per_item, s);
}

template <int NB, auto K>
static cudaError_t launch_small(int64_t tiles, int sm, const GridTable &t, cudaStream_t s) {
    const cudaError_t e = ensure_dyn_smem<K>(static_cast<size_t>(sm));
    if (e != cudaSuccess) return e;
    return launch_pdl(K, dim3(static_cast<unsigned>(tiles)), dim3(NB * kTile), static_cast<size_t>(sm), s, t.desc,
                      t.tmaps, t.n, t.err);
}

// Bands per line (the m2 / m3 banding of Alg. 1): the table's `bands` if set, else four
// (small mode) or four / eight by line length (large mode).  Small mode takes 1, 2, 4 or
// 8 bands, large mode 4 or 8; vedt_map_set_bands admits no other value.
static int bands_for(const GridTable &t, int line) {
    if (t.bands) return t.bands;
    if (!t.large) return kNBY;
    return line <= 256 ? kNBLs : kNBL;
}

cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s) {
    if (t.tiles_y == 0) return cudaSuccess;
    const int nb = bands_for(t, t.maxY);
    if (!t.large) return launch_env_y(t, nb, s);
    if (nb == 4) return launch_small<4, k_pass_y_small<4, true>>(t.tiles_y, small_smem<4, PolY<true>>(t.maxY), t, s);
    return launch_small<8, k_pass_y_small<8, true>>(t.tiles_y, small_smem<8, PolY<true>>(t.maxY), t, s);
}

cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s) {
    if (t.tiles_z == 0) return cudaSuccess;
    const int nb = bands_for(t, t.maxZ);
    if (!t.large) return launch_env_z(t, nb, s);
    const size_t s4 = small_smem<4, PolZ<true>>(t.maxZ), s8 = small_smem<8, PolZ<true>>(t.maxZ);
    if (t.pzx == 8)
        return nb == 4 ? launch_small<4, k_pass_z_small<4, true, 8>>(t.tiles_z, s4, t, s)
                       : launch_small<8, k_pass_z_small<8, true, 8>>(t.tiles_z, s8, t, s);
    if (t.pzx != kCols) return cudaErrorInvalidValue;   // tiles counted for another shape
    return nb == 4 ? launch_small<4, k_pass_z_small<4, true, kCols>>(t.tiles_z, s4, t, s)
                   : launch_small<8, k_pass_z_small<8, true, kCols>>(t.tiles_z, s8, t, s);
}

}  // namespace vedt
