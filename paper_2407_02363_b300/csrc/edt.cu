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
// Passes Y and Z (envelope.cu / envelope.cuh) run one CTA of NB warps per tile of 32
// columns (the m2 / m3 banding of Alg. 1): lane t owns column t, warp b the b-th band of
// every line.  The domination test is exact integer arithmetic with h_s = f(s) + s^2:
//   b (above a) is dropped under c  iff  (h_c - h_b)(b - a) <= (h_b - h_a)(c - b),
// i.e. c overtakes b no later than b overtakes a.
//
// This file holds pass X for every size (k_pass_x_one and k_pass_x_small for grids with
// every dim <= 256: 8-bit row sites and a per-row flag; k_pass_x above: 16-bit row sites,
// 0xFFFF for an empty row, and the row flag), the two persistent batch kernels over the
// envelope tiles, and the launchers of the three passes.
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

// Default bands per line (the m2 / m3 banding of Alg. 1).
constexpr int kNBY = 4;   // grids with every dim <= 256
constexpr int kNBL = 8;   // once some dim exceeds 256: lines over 256 long
constexpr int kNBLs = 4;  // once some dim exceeds 256: lines up to 256 long

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
// tiles with the large word sizes (envelope.cuh, PolYL / PolZL; 32 x 1 pass-Z tiles).  The tile area of shared memory is reused from
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
                if (is_y)
                    lenv::tile_y<2, false, lenv::PolYL>(gd[g], &tm[2 * g], static_cast<int>(t - gd[g].ty_begin), smem,
                                                        &bar, phase, err);
                else
                    lenv::tile_z<2, false, kCols, lenv::PolZL>(gd[g], &tm[2 * g + 1],
                                                               static_cast<int>(t - gd[g].tz_begin), smem, &bar,
                                                               phase, err);
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
    const size_t sy = static_cast<size_t>(lenv::Layout<NB, lenv::PolY>(t.maxY).bytes);
    const size_t sz = static_cast<size_t>(lenv::Layout<NB, lenv::PolZ>(t.maxZ).bytes);
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
    const size_t sy = static_cast<size_t>(lenv::Layout<2, lenv::PolYL>(t.maxY).bytes);
    const size_t sz = static_cast<size_t>(lenv::Layout<2, lenv::PolZL>(t.maxZ).bytes);
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

// Bands per line (the m2 / m3 banding of Alg. 1): the table's `bands` if set, else four
// (small mode) or four / eight by line length (large mode).  Small mode takes 1, 2, 4 or
// 8 bands, large mode 4 or 8; vedt_map_set_bands admits no other value.
static int bands_for(const GridTable &t, int line) {
    if (t.bands) return t.bands;
    if (!t.large) return kNBY;
    return line <= 256 ? kNBLs : kNBL;
}

cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s) { return launch_env_y(t, bands_for(t, t.maxY), s); }

cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s) { return launch_env_z(t, bands_for(t, t.maxZ), s); }

}  // namespace vedt
