// Statistical outlier filter of the raw point cloud (Sec. III-A): each point's mean
// Euclidean distance d_i to its k nearest neighbours; the cloud's mean and standard
// deviation of d_i; a point is kept iff d_i <= mean + std_mul * std.
//
// Exact kNN on a uniform cell grid: the valid points (finite coordinates) are counted into
// cells of edge `cs`, sorted by cell (counting sort: histogram, exclusive scan, scatter),
// and one thread per sorted point searches cubes of cells of growing Chebyshev radius
// around its own cell, keeping its k smallest squared distances in ascending order, until
// the k-th is no farther than the nearest face of the searched cube (so no unexamined
// point can be nearer).  The cell edge only sets the speed.
//
// The decision is reached bit for bit like any independent implementation of the same
// definition: squared distances from float32 coordinates in float64 ((dx^2 + dy^2) +
// dz^2, exact differences), the k square roots summed in ascending order, and the sums
// over the cloud kept exactly as 128-bit fixed-point integers (floor(x * 2^80)), so the
// order in which blocks add them cannot change the threshold.  All float64 steps use
// explicitly rounded intrinsics (no contraction).
#include <cfloat>

#include "vedt_internal.h"

namespace vedt {
namespace sorf {

constexpr int kMaxK = 64;
constexpr int kScan = 4096;      // cells per scan block (1024 threads x 4)
constexpr int kStatBlocks = 256;

struct U128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ U128 add128(U128 a, U128 b) {
    U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}
// floor(x * 2^80) for 0 <= x < 2^40 (the scaling by a power of two is exact)
__device__ __forceinline__ U128 fixed80(double x) {
    const double v = x * 0x1p80;
    U128 r;
    if (v < 0x1p64) {
        r.hi = 0;
        r.lo = __double2ull_rz(v);
    } else {
        r.hi = __double2ull_rz(v * 0x1p-64);
        r.lo = __double2ull_rz(v - static_cast<double>(r.hi) * 0x1p64);   // exact remainder
    }
    return r;
}
// round-to-nearest-even conversion of a 128-bit unsigned integer to double: the top 64
// significant bits with the bits below them folded into a sticky bit, then one rounding
__device__ __forceinline__ double u128_to_double(U128 a) {
    if (a.hi == 0) return __ull2double_rn(a.lo);
    const int sh = 64 - __clzll(static_cast<long long>(a.hi));   // 1..64: bits of hi
    unsigned long long top, rest;
    if (sh == 64) {
        top = a.hi;
        rest = a.lo;
    } else {
        top = (a.hi << (64 - sh)) | (a.lo >> sh);
        rest = a.lo << (64 - sh);
    }
    return scalbn(__ull2double_rn(top | (rest != 0 ? 1ull : 0ull)), sh);
}

// float <-> order-preserving unsigned key (for atomic min / max of floats)
__device__ __forceinline__ unsigned fkey(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float funkey(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

struct Plan {
    unsigned lo_key[3], hi_key[3];   // bounding box of the valid points
    unsigned long long m;            // valid points
    unsigned long long kept;
    float lo[3];
    int gdim[3];
    int ncell;
    unsigned nonempty;               // non-empty cells of the first binning
    double cs;
    U128 S, Q;
    double mean, stddev, thr;
};

__device__ __forceinline__ bool valid_point(float x, float y, float z) {
    return isfinite(x) && isfinite(y) && isfinite(z);
}

__global__ void k_sor_init(Plan *p) {
    for (int a = 0; a < 3; ++a) {
        p->lo_key[a] = 0xFFFFFFFFu;
        p->hi_key[a] = 0u;
    }
    p->m = 0;
    p->kept = 0;
    p->S = p->Q = U128{0, 0};
    p->mean = p->stddev = p->thr = __longlong_as_double(0x7FF8000000000000ll);   // NaN until computed
}

__global__ void __launch_bounds__(256) k_sor_bbox(const float *__restrict__ xyz, int64_t n, Plan *p) {
    unsigned lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
    unsigned cnt = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        if (!valid_point(v[0], v[1], v[2])) continue;
        ++cnt;
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], fkey(v[a]));
            hi[a] = max(hi[a], fkey(v[a]));
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, d);
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], __shfl_down_sync(0xffffffffu, lo[a], d));
            hi[a] = max(hi[a], __shfl_down_sync(0xffffffffu, hi[a], d));
        }
    }
    // one set of atomics per block (the warps' partials meet in shared memory first)
    __shared__ unsigned s_lo[3][8], s_hi[3][8], s_cnt[8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_cnt[w] = cnt;
        for (int a = 0; a < 3; ++a) {
            s_lo[a][w] = lo[a];
            s_hi[a][w] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int u = 1; u < static_cast<int>(blockDim.x >> 5); ++u) {
            cnt += s_cnt[u];
            for (int a = 0; a < 3; ++a) {
                lo[a] = min(lo[a], s_lo[a][u]);
                hi[a] = max(hi[a], s_hi[a][u]);
            }
        }
        if (cnt) {
            atomicAdd(&p->m, static_cast<unsigned long long>(cnt));
            for (int a = 0; a < 3; ++a) {
                atomicMin(&p->lo_key[a], lo[a]);
                atomicMax(&p->hi_key[a], hi[a]);
            }
        }
    }
}

// grid of cell edge cs over the box (cs grown until there are at most `cap` cells)
__device__ void set_grid(Plan *p, const double (&ext)[3], double cs, int cap) {
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) cells *= floor(ext[a] / cs) + 1.0;
        if (cells <= cap) break;
        cs *= 1.25;
    }
    for (int a = 0; a < 3; ++a) p->gdim[a] = static_cast<int>(floor(ext[a] / cs)) + 1;
    p->ncell = p->gdim[0] * p->gdim[1] * p->gdim[2];
    p->cs = cs;
}

// Cell edge from the box: cs = sqrt(A k / (pi m)) with A the sum of the box's three face
// areas, i.e. about k points within one cell edge for a cloud spread over surfaces of that
// area; grown until the grid has at most `cap` cells.
__global__ void k_sor_plan(Plan *p, int k, int cap) {
    if (p->m == 0) {
        p->ncell = 0;
        return;
    }
    double ext[3], emax = 0.0;
    for (int a = 0; a < 3; ++a) {
        p->lo[a] = funkey(p->lo_key[a]);
        ext[a] = static_cast<double>(funkey(p->hi_key[a])) - static_cast<double>(p->lo[a]);
        emax = fmax(emax, ext[a]);
    }
    const double area = ext[0] * ext[1] + ext[1] * ext[2] + ext[0] * ext[2];
    double cs = sqrt(area * k / (3.141592653589793 * static_cast<double>(p->m)));
    cs = fmax(cs, emax * 1e-6);
    if (!(cs > 0.0)) cs = 1.0;   // every valid point at one position
    p->nonempty = 0;
    set_grid(p, ext, cs, cap);
}

// Second cell edge from the first binning: points per non-empty cell rho estimates the
// surface density times cs^2, and cs' = 1.2 cs sqrt(k / (pi rho)) puts about k points
// within one cell edge of a point on such a surface.
__global__ void __launch_bounds__(256) k_sor_nonempty(const unsigned *__restrict__ count, int n, Plan *p) {
    unsigned c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += count[i] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&p->nonempty, c);
}

__global__ void k_sor_replan(Plan *p, int k, int cap) {
    if (p->m == 0 || p->nonempty == 0) return;
    const double rho = static_cast<double>(p->m) / p->nonempty;
    double ext[3];
    for (int a = 0; a < 3; ++a) ext[a] = static_cast<double>(funkey(p->hi_key[a])) - static_cast<double>(p->lo[a]);
    double cs = 1.2 * p->cs * sqrt(k / (3.141592653589793 * rho));
    double emax = fmax(ext[0], fmax(ext[1], ext[2]));
    cs = fmax(cs, emax * 1e-6);
    if (!(cs > 0.0)) cs = 1.0;
    set_grid(p, ext, cs, cap);
}

__device__ __forceinline__ int cell_coord(float v, float lo, double cs, int g) {
    const int c = static_cast<int>(floor((static_cast<double>(v) - static_cast<double>(lo)) / cs));
    return min(max(c, 0), g - 1);
}

__global__ void __launch_bounds__(256) k_sor_count(const float *__restrict__ xyz, int64_t n, const Plan *p,
                                                   unsigned *__restrict__ count, int *__restrict__ cell_of,
                                                   unsigned *__restrict__ rank) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const double cs = p->cs;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!valid_point(x, y, z)) {
            cell_of[i] = -1;
            continue;
        }
        const int c = cell_coord(x, p->lo[0], cs, p->gdim[0]) +
                      p->gdim[0] * (cell_coord(y, p->lo[1], cs, p->gdim[1]) +
                                    p->gdim[1] * cell_coord(z, p->lo[2], cs, p->gdim[2]));
        cell_of[i] = c;
        rank[i] = atomicAdd(count + c, 1u);
    }
}

// exclusive scan of count[0 .. n) into start (n <= kScan * kScan), three launches
__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned *__restrict__ in, unsigned *__restrict__ out,
                                                      unsigned *__restrict__ sums, int n) {
    __shared__ unsigned s[1024];
    const int base = blockIdx.x * kScan + threadIdx.x * 4;
    unsigned v[4], t = 0;
    for (int j = 0; j < 4; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        t += v[j];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // inclusive Hillis-Steele over the thread totals
        const unsigned u = threadIdx.x >= d ? s[threadIdx.x - d] : 0u;
        __syncthreads();
        s[threadIdx.x] += u;
        __syncthreads();
    }
    unsigned run = s[threadIdx.x] - t;
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 1023) sums[blockIdx.x] = s[1023];
}

__global__ void __launch_bounds__(1024) k_scan_sums(unsigned *__restrict__ sums, int nb) {
    __shared__ unsigned s[kScan];
    for (int j = threadIdx.x; j < kScan; j += 1024) s[j] = j < nb ? sums[j] : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int j = 0; j < nb; ++j) {
            const unsigned t = s[j];
            s[j] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += 1024) sums[j] = s[j];
}

__global__ void __launch_bounds__(1024) k_scan_add(unsigned *__restrict__ out, const unsigned *__restrict__ sums, int n) {
    const int base = blockIdx.x * kScan + threadIdx.x * 4;
    const unsigned add = sums[blockIdx.x];
    for (int j = 0; j < 4; ++j)
        if (base + j < n) out[base + j] += add;
}

// sorted[start[cell] + rank] = (x, y, z, original index)
__global__ void __launch_bounds__(256) k_sor_scatter(const float *__restrict__ xyz, int64_t n,
                                                     const int *__restrict__ cell_of, const unsigned *__restrict__ rank,
                                                     const unsigned *__restrict__ start, float4 *__restrict__ sorted) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cell_of[i];
        if (c < 0) continue;
        sorted[start[c] + rank[i]] =
            make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __int_as_float(static_cast<int>(i)));
    }
}

__device__ __forceinline__ double sq_dist(float4 a, float4 b) {
    const double dx = __dadd_rn(static_cast<double>(a.x), -static_cast<double>(b.x));
    const double dy = __dadd_rn(static_cast<double>(a.y), -static_cast<double>(b.y));
    const double dz = __dadd_rn(static_cast<double>(a.z), -static_cast<double>(b.z));
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// One thread per sorted point (neighbouring threads share cells): the mean distance to
// its kk = min(k, m - 1) nearest valid points, written at the point's original index.
//
// The search keeps the L = kk + kExtra candidates with the smallest float32 squared
// distance in a max-heap of packed (float32 bits << 32 | sorted slot) keys in shared
// memory (column threadIdx.x of heap[L][kKnnThreads]); non-negative float bits order like
// the floats.  A float32 squared distance is within a relative 3e-7 plus an absolute 1e-44
// (subnormal squares) of the float64 one, so with tau the kk-th smallest float32 value,
// every one of the kk nearest by float64 has a float32 value <= tau (1 + 4e-6) + 1e-40:
// they are all in the heap unless more than kExtra candidates share that band, in which
// case the searched cube is scanned again in float64 over the band.  The ring search
// stops once the heap's largest float32 value times (1 + 1e-5), plus 1e-39, lies within
// the squared distance to the searched cube's nearest open face, which keeps every
// unexamined point out of the band.
constexpr int kKnnThreads = 128;
constexpr int kExtra = 4;
constexpr float kBand = 1.000004f;
constexpr float kStop = 1.00001f;

__device__ __forceinline__ unsigned long long hkey(float v, unsigned t) {
    return (static_cast<unsigned long long>(__float_as_uint(v)) << 32) | t;
}
// max-heap over h[0 .. n) (stride kKnnThreads)
__device__ __forceinline__ void heap_up(unsigned long long *h, int j) {
    const unsigned long long x = h[j * kKnnThreads];
    while (j > 0) {
        const int pj = (j - 1) >> 1;
        const unsigned long long y = h[pj * kKnnThreads];
        if (y >= x) break;
        h[j * kKnnThreads] = y;
        j = pj;
    }
    h[j * kKnnThreads] = x;
}
__device__ __forceinline__ void heap_down(unsigned long long *h, int n, unsigned long long x) {
    int j = 0;
    for (;;) {
        int c = 2 * j + 1;
        if (c >= n) break;
        unsigned long long y = h[c * kKnnThreads];
        if (c + 1 < n) {
            const unsigned long long z = h[(c + 1) * kKnnThreads];
            if (z > y) {
                y = z;
                ++c;
            }
        }
        if (y <= x) break;
        h[j * kKnnThreads] = y;
        j = c;
    }
    h[j * kKnnThreads] = x;
}

__device__ __forceinline__ float f32_sq(const float4 &a, const float4 &b) {
    const float fx = a.x - b.x, fy = a.y - b.y, fz = a.z - b.z;
    return fx * fx + fy * fy + fz * fz;
}

// Visits every candidate of the cells at Chebyshev distance r from c (the shell).
template <class F>
__device__ __forceinline__ void for_shell(const int (&c)[3], const int (&g)[3], int r,
                                          const unsigned *__restrict__ start, F &&f) {
    for (int dz = -r; dz <= r; ++dz) {
        const int cz = c[2] + dz;
        if (cz < 0 || cz >= g[2]) continue;
        for (int dy = -r; dy <= r; ++dy) {
            const int cy = c[1] + dy;
            if (cy < 0 || cy >= g[1]) continue;
            const bool inner = (dz > -r && dz < r && dy > -r && dy < r);
            for (int dx = -r; dx <= r; dx += (inner ? 2 * r : 1)) {
                const int cx = c[0] + dx;
                if (cx >= 0 && cx < g[0]) {
                    const int cell = cx + g[0] * (cy + g[1] * cz);
                    const unsigned e = start[cell + 1];
                    for (unsigned t = start[cell]; t < e; ++t) f(t);
                }
                if (r == 0) break;
            }
        }
    }
}

__global__ void __launch_bounds__(kKnnThreads) k_sor_knn(const float4 *__restrict__ sorted,
                                                         const unsigned *__restrict__ start,
                                                         const Plan *__restrict__ p, int k, double *__restrict__ d_out) {
    extern __shared__ unsigned long long sheap[];
    const unsigned long long m = p->m;
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (static_cast<unsigned long long>(s) >= m) return;
    unsigned long long *h = sheap + threadIdx.x;   // entry j at h[j * kKnnThreads]
    const float4 q = sorted[s];
    const int i = __float_as_int(q.w);
    const int kk = static_cast<int>(min(static_cast<unsigned long long>(k), m - 1));
    if (kk == 0) {
        d_out[i] = 0.0;
        return;
    }
    const int L = kk + kExtra;
    const int g[3] = {p->gdim[0], p->gdim[1], p->gdim[2]};
    const double cs = p->cs;
    const float lo[3] = {p->lo[0], p->lo[1], p->lo[2]};
    const float qv[3] = {q.x, q.y, q.z};
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_coord(qv[a], lo[a], cs, g[a]);
    // margin for the rounding of the cell assignment (float64 on float32 coordinates)
    const double margin = cs * 1e-9;
    int cnt = 0, rmax = 0;
    bool self_seen = false;
    auto is_self = [&](const float4 &o) {   // the point itself, or one equal copy of it
        if (!self_seen && o.x == q.x && o.y == q.y && o.z == q.z) {
            self_seen = true;
            return true;
        }
        return false;
    };
    for (int r = 0;; ++r) {
        rmax = r;
        for_shell(c, g, r, start, [&](unsigned t) {
            const float4 o = sorted[t];
            if (is_self(o)) return;
            const unsigned long long key = hkey(f32_sq(q, o), t);
            if (cnt < L) {
                h[cnt * kKnnThreads] = key;
                heap_up(h, cnt++);
            } else if (key < h[0]) {
                heap_down(h, L, key);
            }
        });
        // distance from q to the nearest face of the searched cube that has cells beyond it
        double bound = DBL_MAX;
        bool whole = true;
        for (int a = 0; a < 3; ++a) {
            if (c[a] - r > 0) {
                whole = false;
                bound = fmin(bound, static_cast<double>(qv[a]) - (static_cast<double>(lo[a]) + (c[a] - r) * cs));
            }
            if (c[a] + r < g[a] - 1) {
                whole = false;
                bound = fmin(bound, static_cast<double>(lo[a]) + (c[a] + r + 1) * cs - static_cast<double>(qv[a]));
            }
        }
        if (whole) break;
        bound = fmax(bound - margin, 0.0);
        if (cnt == L) {
            const double top = static_cast<double>(__uint_as_float(static_cast<unsigned>(h[0] >> 32)));
            if (top * kStop + 1e-39 <= bound * bound) break;
        }
    }
    // heap sort: ascending keys in h[0 .. cnt)
    for (int n = cnt; n > 1; --n) {
        const unsigned long long top = h[0];
        heap_down(h, n - 1, h[(n - 1) * kKnnThreads]);
        h[(n - 1) * kKnnThreads] = top;
    }
    const float tau = __uint_as_float(static_cast<unsigned>(h[(kk - 1) * kKnnThreads] >> 32));
    const float band = tau * kBand + 1e-40f;
    int nb = kk;   // entries in the band: h[0 .. nb)
    while (nb < cnt && __uint_as_float(static_cast<unsigned>(h[nb * kKnnThreads] >> 32)) <= band) ++nb;
    double acc = 0.0;
    if (nb < L || cnt < L) {
        // the band is complete in the heap: float64 values of its entries, sorted
        for (int j = 0; j < nb; ++j) {
            const double v = sq_dist(q, sorted[static_cast<unsigned>(h[j * kKnnThreads])]);
            h[j * kKnnThreads] = static_cast<unsigned long long>(__double_as_longlong(v));
        }
        for (int j = 1; j < nb; ++j) {   // nearly sorted already
            const unsigned long long x = h[j * kKnnThreads];
            int u = j;
            while (u > 0 && h[(u - 1) * kKnnThreads] > x) {
                h[u * kKnnThreads] = h[(u - 1) * kKnnThreads];
                --u;
            }
            h[u * kKnnThreads] = x;
        }
    } else {
        // more than kExtra candidates share the band: float64 over the band of the whole
        // searched cube, the kk smallest in a max-heap of float64 bits
        int n64 = 0;
        self_seen = false;
        for (int r = 0; r <= rmax; ++r)
            for_shell(c, g, r, start, [&](unsigned t) {
                const float4 o = sorted[t];
                if (is_self(o) || f32_sq(q, o) > band) return;
                const unsigned long long v = static_cast<unsigned long long>(__double_as_longlong(sq_dist(q, o)));
                if (n64 < kk) {
                    h[n64 * kKnnThreads] = v;
                    heap_up(h, n64++);
                } else if (v < h[0]) {
                    heap_down(h, kk, v);
                }
            });
        for (int n = kk; n > 1; --n) {
            const unsigned long long top = h[0];
            heap_down(h, n - 1, h[(n - 1) * kKnnThreads]);
            h[(n - 1) * kKnnThreads] = top;
        }
    }
    for (int t = 0; t < kk; ++t) acc = __dadd_rn(acc, __dsqrt_rn(__longlong_as_double(static_cast<long long>(h[t * kKnnThreads]))));
    d_out[i] = __ddiv_rn(acc, static_cast<double>(kk));
}

// per-block exact sums of floor(d * 2^80) and floor(d^2 * 2^80) over the valid points
__global__ void __launch_bounds__(256) k_sor_sums(const double *__restrict__ d, const int *__restrict__ cell_of,
                                                  int64_t n, U128 *__restrict__ part) {
    __shared__ U128 sS[256], sQ[256];
    U128 S{0, 0}, Q{0, 0};
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (cell_of[i] < 0) continue;
        const double v = d[i];
        S = add128(S, fixed80(v));
        Q = add128(Q, fixed80(__dmul_rn(v, v)));
    }
    sS[threadIdx.x] = S;
    sQ[threadIdx.x] = Q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sS[threadIdx.x] = add128(sS[threadIdx.x], sS[threadIdx.x + w]);
            sQ[threadIdx.x] = add128(sQ[threadIdx.x], sQ[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sS[0];
        part[2 * blockIdx.x + 1] = sQ[0];
    }
}

__global__ void __launch_bounds__(kStatBlocks) k_sor_threshold(const U128 *__restrict__ part, Plan *p, double std_mul) {
    __shared__ U128 sS[kStatBlocks], sQ[kStatBlocks];
    sS[threadIdx.x] = part[2 * threadIdx.x];
    sQ[threadIdx.x] = part[2 * threadIdx.x + 1];
    __syncthreads();
    for (int w = kStatBlocks / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sS[threadIdx.x] = add128(sS[threadIdx.x], sS[threadIdx.x + w]);
            sQ[threadIdx.x] = add128(sQ[threadIdx.x], sQ[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const U128 S = sS[0], Q = sQ[0];
    p->S = S;
    p->Q = Q;
    const double m = static_cast<double>(p->m);
    const double s = u128_to_double(S) * 0x1p-80, q = u128_to_double(Q) * 0x1p-80;
    const double mean = __ddiv_rn(s, m);
    double var = 0.0;
    if (p->m > 1) var = __ddiv_rn(__dadd_rn(q, -__ddiv_rn(__dmul_rn(s, s), m)), m - 1.0);
    var = fmax(var, 0.0);
    const double sd = __dsqrt_rn(var);
    p->mean = mean;
    p->stddev = sd;
    p->thr = __dadd_rn(mean, __dmul_rn(std_mul, sd));
}

__global__ void __launch_bounds__(256) k_sor_keep(const double *__restrict__ d, const int *__restrict__ cell_of,
                                                  int64_t n, Plan *p, uint8_t *__restrict__ keep) {
    const double thr = p->thr;
    unsigned kept = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const bool k = cell_of[i] >= 0 && d[i] <= thr;
        keep[i] = k ? 1 : 0;
        kept += k;
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(0xffffffffu, kept, o);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&p->kept, static_cast<unsigned long long>(kept));
}

}  // namespace sorf
}  // namespace vedt

using namespace vedt;
using namespace vedt::sorf;

struct vedt_sor {
    int64_t cap = 0;        // points
    int cell_cap = 0;       // cells
    cudaStream_t stream = nullptr;
    Plan *plan = nullptr;
    unsigned *count = nullptr, *start = nullptr, *sums = nullptr, *rank = nullptr;
    int *cell_of = nullptr;
    float4 *sorted = nullptr;
    double *d = nullptr;
    U128 *part = nullptr;
};

namespace {
void free_sor(vedt_sor *f) {
    cudaFree(f->plan);
    cudaFree(f->count);
    cudaFree(f->start);
    cudaFree(f->sums);
    cudaFree(f->rank);
    cudaFree(f->cell_of);
    cudaFree(f->sorted);
    cudaFree(f->d);
    cudaFree(f->part);
    delete f;
}
int sms() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}
}  // namespace

extern "C" {

vedt_status vedt_sor_create(int64_t max_points, void *stream, vedt_sor **out) {
    if (!out || max_points < 1 || max_points > (int64_t(1) << 31) - 1) return VEDT_EINVAL;
    *out = nullptr;
    vedt_sor *f = new (std::nothrow) vedt_sor();
    if (!f) return VEDT_ENOMEM;
    f->cap = max_points;
    const int64_t cells = std::min<int64_t>(std::max<int64_t>(2 * max_points, 1 << 16), int64_t(kScan) * kScan - 1);
    f->cell_cap = static_cast<int>(cells);
    f->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&f->plan, sizeof(Plan));
    if (e == cudaSuccess) e = cudaMalloc(&f->count, sizeof(unsigned) * (cells + 1));
    if (e == cudaSuccess) e = cudaMalloc(&f->start, sizeof(unsigned) * (cells + 1));
    if (e == cudaSuccess) e = cudaMalloc(&f->sums, sizeof(unsigned) * kScan);
    if (e == cudaSuccess) e = cudaMalloc(&f->rank, sizeof(unsigned) * max_points);
    if (e == cudaSuccess) e = cudaMalloc(&f->cell_of, sizeof(int) * max_points);
    if (e == cudaSuccess) e = cudaMalloc(&f->sorted, sizeof(float4) * max_points);
    if (e == cudaSuccess) e = cudaMalloc(&f->d, sizeof(double) * max_points);
    if (e == cudaSuccess) e = cudaMalloc(&f->part, sizeof(U128) * 2 * kStatBlocks);
    if (e != cudaSuccess) {
        free_sor(f);
        return e == cudaErrorMemoryAllocation ? VEDT_ENOMEM : VEDT_ECUDA;
    }
    *out = f;
    return VEDT_OK;
}

vedt_status vedt_sor_destroy(vedt_sor *f) {
    if (!f) return VEDT_OK;
    cudaStreamSynchronize(f->stream);
    free_sor(f);
    return VEDT_OK;
}

vedt_status vedt_sor_filter(vedt_sor *f, const float *xyz_dev, int64_t n, int k, double std_mul,
                            uint8_t *keep_dev) {
    if (!f || n < 0 || n > f->cap || k < 1 || k > kMaxK || !std::isfinite(std_mul) ||
        (n > 0 && (!xyz_dev || !keep_dev)))
        return VEDT_EINVAL;
    cudaStream_t s = f->stream;
    k_sor_init<<<1, 1, 0, s>>>(f->plan);
    if (n == 0) return cudaGetLastError() == cudaSuccess ? VEDT_OK : VEDT_ECUDA;
    const int cap_blocks = sms() * 8;
    const int nb = static_cast<int>(std::min<int64_t>((n + 255) / 256, cap_blocks));
    k_sor_bbox<<<nb, 256, 0, s>>>(xyz_dev, n, f->plan);
    k_sor_plan<<<1, 1, 0, s>>>(f->plan, k, f->cell_cap);
    // the histogram and the scan run over the whole cell capacity (the grid's cell count
    // is known on the device only); unused cells stay empty
    const int ncs = f->cell_cap + 1;
    if (cudaMemsetAsync(f->count, 0, sizeof(unsigned) * ncs, s) != cudaSuccess) return VEDT_ECUDA;
    k_sor_count<<<nb, 256, 0, s>>>(xyz_dev, n, f->plan, f->count, f->cell_of, f->rank);
    // refine the cell edge from the first binning's occupancy, then bin again
    k_sor_nonempty<<<cap_blocks, 256, 0, s>>>(f->count, f->cell_cap, f->plan);
    k_sor_replan<<<1, 1, 0, s>>>(f->plan, k, f->cell_cap);
    if (cudaMemsetAsync(f->count, 0, sizeof(unsigned) * ncs, s) != cudaSuccess) return VEDT_ECUDA;
    k_sor_count<<<nb, 256, 0, s>>>(xyz_dev, n, f->plan, f->count, f->cell_of, f->rank);
    const int sb = (ncs + kScan - 1) / kScan;
    k_scan_blocks<<<sb, 1024, 0, s>>>(f->count, f->start, f->sums, ncs);
    k_scan_sums<<<1, 1024, 0, s>>>(f->sums, sb);
    k_scan_add<<<sb, 1024, 0, s>>>(f->start, f->sums, ncs);
    k_sor_scatter<<<nb, 256, 0, s>>>(xyz_dev, n, f->cell_of, f->rank, f->start, f->sorted);
    const size_t knn_smem = sizeof(unsigned long long) * (k + kExtra) * kKnnThreads;
    if (ensure_dyn_smem<k_sor_knn>(knn_smem) != cudaSuccess) return VEDT_ECUDA;
    k_sor_knn<<<static_cast<unsigned>((n + kKnnThreads - 1) / kKnnThreads), kKnnThreads, knn_smem, s>>>(
        f->sorted, f->start, f->plan, k, f->d);
    k_sor_sums<<<kStatBlocks, 256, 0, s>>>(f->d, f->cell_of, n, f->part);
    k_sor_threshold<<<1, kStatBlocks, 0, s>>>(f->part, f->plan, std_mul);
    k_sor_keep<<<nb, 256, 0, s>>>(f->d, f->cell_of, n, f->plan, keep_dev);
    return cudaGetLastError() == cudaSuccess ? VEDT_OK : VEDT_ECUDA;
}

vedt_status vedt_sor_stats(vedt_sor *f, double stats_out[3], int64_t counts_out[2]) {
    if (!f) return VEDT_EINVAL;
    if (cudaStreamSynchronize(f->stream) != cudaSuccess) return VEDT_ECUDA;
    Plan p;
    if (cudaMemcpy(&p, f->plan, sizeof(Plan), cudaMemcpyDeviceToHost) != cudaSuccess) return VEDT_ECUDA;
    if (stats_out) {
        stats_out[0] = p.mean;
        stats_out[1] = p.stddev;
        stats_out[2] = p.thr;
    }
    if (counts_out) {
        counts_out[0] = static_cast<int64_t>(p.m);
        counts_out[1] = static_cast<int64_t>(p.kept);
    }
    return VEDT_OK;
}

vedt_status vedt_sor_mean_distances(vedt_sor *f, const double **d_dev) {
    if (!f || !d_dev) return VEDT_EINVAL;
    *d_dev = f->d;
    return VEDT_OK;
}

}  // extern "C"
