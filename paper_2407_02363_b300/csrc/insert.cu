// Per-frame occupancy updates and the sphere query (Alg. 2 lines 4-7 and 10).
//
// All floating-point steps that decide an integer voxel use explicitly rounded
// intrinsics in a fixed order (no FMA contraction, IEEE division), so that a point lands
// in the same voxel as under any other correctly rounded fp32 evaluation of
//   w_a = ((R_a0 p_x + R_a1 p_y) + R_a2 p_z) + t_a,   v_a = floor((w_a - origin_a) / vs).
#include "vedt_internal.h"

namespace vedt {

struct Origin { float o[3]; };

// ClearMap (Alg. 2 line 4): 16-byte stores over the byte grid, byte tail.
__global__ void __launch_bounds__(256) k_clear(uint8_t *__restrict__ p, int64_t n) {
    pdl_trigger();
    pdl_wait();
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const int64_t head = static_cast<int64_t>(((a + 15) & ~uintptr_t(15)) - a);
    const int64_t h = head < n ? head : n;
    const int64_t nvec = (n - h) >> 4;
    uint4 *v = reinterpret_cast<uint4 *>(p + h);
    int64_t i = tid;
    for (; i + 3 * stride < nvec; i += 4 * stride) {   // four independent 16-byte stores in flight
        v[i] = make_uint4(0, 0, 0, 0);
        v[i + stride] = make_uint4(0, 0, 0, 0);
        v[i + 2 * stride] = make_uint4(0, 0, 0, 0);
        v[i + 3 * stride] = make_uint4(0, 0, 0, 0);
    }
    for (; i < nvec; i += stride) v[i] = make_uint4(0, 0, 0, 0);
    for (int64_t i = tid; i < h; i += stride) p[i] = 0;
    for (int64_t i = h + (nvec << 4) + tid; i < n; i += stride) p[i] = 0;
}

// Change detection of incremental maps: compares grid blockIdx.y's occupancy (n_al bytes,
// 16-byte words) with the snapshot taken at its last EDT, refreshes the snapshot where
// they differ and sets changed[grid] (zeroed before the launch) if any byte differed.
__global__ void __launch_bounds__(256) k_occ_diff(const uint8_t *__restrict__ occ, uint8_t *__restrict__ snap,
                                                  uint32_t *__restrict__ changed, int64_t n_al) {
    pdl_trigger();
    pdl_wait();
    const int g = blockIdx.y;
    const uint4 *o = reinterpret_cast<const uint4 *>(occ + g * n_al);
    uint4 *sp = reinterpret_cast<uint4 *>(snap + g * n_al);
    const int64_t nvec = n_al >> 4;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int diff = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec; i += stride) {
        const uint4 a = o[i], b = sp[i];
        if (a.x != b.x || a.y != b.y || a.z != b.z || a.w != b.w) {
            sp[i] = a;
            diff = 1;
        }
    }
    if (__syncthreads_or(diff) && threadIdx.x == 0) changed[g] = 1u;
}

// Bayesian occupancy update of M_I (Sec. III-A, log-odds form): per voxel, a hit (some
// point of the frame landed in it) adds l_hit, a miss subtracts l_miss, the sum is
// clamped to [l_min, l_max], and the voxel is occupied for the EDT iff it reaches the
// threshold.  16 voxels per thread and iteration; the alignment tail past the n voxels
// keeps its zeros.

__global__ void __launch_bounds__(256) k_logodds(uint8_t *__restrict__ occ, int8_t *__restrict__ L, int64_t n,
                                                 LogOdds p) {
    const int64_t nvec = (n + 15) / 16;
    pdl_trigger();
    pdl_wait();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    uint4 *o4 = reinterpret_cast<uint4 *>(occ);
    uint4 *l4 = reinterpret_cast<uint4 *>(L);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec; i += stride) {
        uint4 ov = o4[i], lv = l4[i];
        uint8_t *ob = reinterpret_cast<uint8_t *>(&ov);
        int8_t *lb = reinterpret_cast<int8_t *>(&lv);
        const int64_t left = n - i * 16;
        const int valid = left < 16 ? static_cast<int>(left) : 16;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            if (b < valid) {
                const int v = logodds_step(lb[b], ob[b] != 0, p);
                lb[b] = static_cast<int8_t>(v);
                ob[b] = v >= p.thr ? 1 : 0;
            }
        }
        o4[i] = ov;
        l4[i] = lv;
    }
}

struct Pose12 { float T[12]; };

// Insert(Point_Cloud) with robot-point removal (Alg. 2 line 7; Sec. III-A).
__global__ void __launch_bounds__(256) k_insert_points(uint8_t *__restrict__ env, const uint8_t *__restrict__ self,
                                                       int X, int Y, int Z, float vs, Origin org,
                                                       const float *__restrict__ xyz, int64_t n, Pose12 T, int use_T,
                                                       int filter_self, const uint8_t *__restrict__ keep,
                                                       unsigned long long *counts) {
    pdl_trigger();
    pdl_wait();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned long long written = 0, outside = 0, filtered = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (keep && !keep[i]) continue;   // dropped by the outlier filter
        float wx = __ldg(xyz + 3 * i), wy = __ldg(xyz + 3 * i + 1), wz = __ldg(xyz + 3 * i + 2);
        if (use_T) rigid(T.T, wx, wy, wz, wx, wy, wz);
        int vx, vy, vz;
        if (!voxel_coord(wx, org.o[0], vs, X, vx) || !voxel_coord(wy, org.o[1], vs, Y, vy) ||
            !voxel_coord(wz, org.o[2], vs, Z, vz)) {
            ++outside;
            continue;
        }
        const int64_t id = vx + static_cast<int64_t>(X) * (vy + static_cast<int64_t>(Y) * vz);
        if (filter_self && self[id]) {
            ++filtered;
            continue;
        }
        env[id] = 1;
        ++written;
    }
    if (counts) {
        // warp-aggregated counters
        for (int d = 16; d > 0; d >>= 1) {
            written += __shfl_down_sync(0xffffffffu, written, d);
            outside += __shfl_down_sync(0xffffffffu, outside, d);
            filtered += __shfl_down_sync(0xffffffffu, filtered, d);
        }
        if ((threadIdx.x & 31) == 0) {
            if (written) atomicAdd(counts + 0, written);
            if (outside) atomicAdd(counts + 1, outside);
            if (filtered) atomicAdd(counts + 2, filtered);
        }
    }
}

// UpdateLinks + Insert(O_Lk) (Alg. 2 lines 5-6): every registered link point is moved by
// its link's pose and marked in the self map if its link is in the mask.  The link points
// and their link indices are copied to the device when the links are registered, before
// any frame, and the poses are launch parameters: a thread loads and places its first
// point before the dependency wait (overlapping the tail of the clear before it) and only
// the store into the self map follows the wait.
__device__ __forceinline__ int64_t link_voxel(const float *__restrict__ pts, const uint8_t *__restrict__ link_of,
                                              int64_t i, const LinkPose &poses, uint32_t mask, int X, int Y, int Z,
                                              float vs, const Origin &org) {
    const int k = link_of[i];
    if (!((mask >> k) & 1u)) return -1;
    float wx, wy, wz;
    rigid(poses.T[k], __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2), wx, wy, wz);
    int vx, vy, vz;
    if (!voxel_coord(wx, org.o[0], vs, X, vx) || !voxel_coord(wy, org.o[1], vs, Y, vy) ||
        !voxel_coord(wz, org.o[2], vs, Z, vz))
        return -1;
    return vx + static_cast<int64_t>(X) * (vy + static_cast<int64_t>(Y) * vz);
}

__global__ void __launch_bounds__(256) k_insert_links(uint8_t *__restrict__ self, int X, int Y, int Z, float vs,
                                                      Origin org, const float *__restrict__ pts,
                                                      const uint8_t *__restrict__ link_of, int64_t n,
                                                      LinkPose poses, uint32_t mask) {
    pdl_trigger();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t first = i < n ? link_voxel(pts, link_of, i, poses, mask, X, Y, Z, vs, org) : -1;
    pdl_wait();   // the self map is cleared by the previous kernel
    if (first >= 0) self[first] = 1;
    for (i += stride; i < n; i += stride) {
        const int64_t id = link_voxel(pts, link_of, i, poses, mask, X, Y, Z, vs, org);
        if (id >= 0) self[id] = 1;
    }
}

// ExtractClosestObstaclePose + Eq. (dist): thread (grid g, sphere i).
__global__ void __launch_bounds__(128) k_query(const QueryGrid *__restrict__ grids, int ng, int X, int Y, int Z,
                                               float vs, Origin org, const float *__restrict__ centres,
                                               const float *__restrict__ radii, int m,
                                               vedt_sphere_result *__restrict__ out) {
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * ng) return;
    const int g = t / m, i = t - g * m;
    // The sphere inputs and the grids' descriptors are written by the host (or by the
    // caller's work before the frame's first kernel, which cannot start until that work
    // has finished), not by the kernels this one waits for: read them before the wait,
    // so that only the field loads follow it.
    const float cx = centres[3 * i], cy = centres[3 * i + 1], cz = centres[3 * i + 2], rad = radii[i];
    const int32_t *sqp = grids[g].sqdist, *ixp = grids[g].idx;
    vedt_sphere_result r;
    int v[3];
    const bool inside = voxel_coord(cx, org.o[0], vs, X, v[0]) && voxel_coord(cy, org.o[1], vs, Y, v[1]) &&
                        voxel_coord(cz, org.o[2], vs, Z, v[2]);
    pdl_wait();   // the fields come from the EDT passes; the results buffer may have been read before
    if (!inside) {
        r.sqdist = -1;
        r.idx = -1;
        r.dist = __int_as_float(0x7fc00000);
        r.clearance = r.dist;
        r.nearest[0] = r.nearest[1] = r.nearest[2] = r.dist;
        r.status = VEDT_SPHERE_OUTSIDE;
        out[t] = r;
        return;
    }
    const int64_t id = v[0] + static_cast<int64_t>(X) * (v[1] + static_cast<int64_t>(Y) * v[2]);
    r.sqdist = sqp[id];
    r.idx = ixp[id];
    if (r.idx < 0) {
        r.dist = __int_as_float(0x7f800000);
        r.clearance = r.dist;
        r.nearest[0] = r.nearest[1] = r.nearest[2] = __int_as_float(0x7fc00000);
        r.status = VEDT_SPHERE_EMPTY;
        out[t] = r;
        return;
    }
    r.dist = __fmul_rn(vs, __fsqrt_rn(static_cast<float>(r.sqdist)));
    r.clearance = __fsub_rn(r.dist, rad);
    const int j = r.idx;
    const int nv[3] = {j % X, (j / X) % Y, j / (X * Y)};
    for (int a = 0; a < 3; ++a)
        r.nearest[a] = __fadd_rn(org.o[a], __fmul_rn(__fadd_rn(static_cast<float>(nv[a]), 0.5f), vs));
    r.status = VEDT_SPHERE_OK;
    out[t] = r;
}


int sm_count() {
    // the launchers ask on every launch: remember the answer per device
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const bool keep = dev >= 0 && dev < kMaxDevices;
    if (keep) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (keep) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

cudaError_t launch_clear(uint8_t *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n / 16 + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int blocks = static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
    return launch_pdl(k_clear, dim3(blocks), dim3(256), 0, s, p, n);
}

cudaError_t launch_logodds(uint8_t *occ, int8_t *L, int64_t n, const int (&p)[5], cudaStream_t s) {
    const int64_t nvec = (n + 15) / 16;
    const int64_t want = (nvec + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8;
    const int blocks = static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
    return launch_pdl(k_logodds, dim3(blocks), dim3(256), 0, s, occ, L, n, LogOdds{p[0], p[1], p[2], p[3], p[4]});
}

cudaError_t launch_occ_diff(const uint8_t *occ, uint8_t *snap, uint32_t *changed, int64_t n_al, int grids,
                            cudaStream_t s) {
    if (n_al <= 0 || grids < 1) return cudaSuccess;
    const int64_t want = (n_al / 16 + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 8 / grids;
    const int blocks = static_cast<int>(want < 1 ? 1 : (want < cap ? want : (cap < 1 ? 1 : cap)));
    return launch_pdl(k_occ_diff, dim3(blocks, grids), dim3(256), 0, s, occ, snap, changed, n_al);
}

cudaError_t launch_insert_points(uint8_t *env, const uint8_t *self, int X, int Y, int Z, float vs,
                                 const float *origin, const float *xyz, int64_t n, const float *T,
                                 int filter_self, const uint8_t *keep, int64_t *counts, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    Origin o{{origin[0], origin[1], origin[2]}};
    Pose12 P{};
    if (T)
        for (int i = 0; i < 12; ++i) P.T[i] = T[i];
    const int64_t want = (n + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int blocks = static_cast<int>(want < cap ? want : cap);
    return launch_pdl(k_insert_points, dim3(blocks), dim3(256), 0, s, env, self, X, Y, Z, vs, o, xyz, n, P,
                      T != nullptr ? 1 : 0, filter_self, keep, reinterpret_cast<unsigned long long *>(counts));
}

cudaError_t launch_insert_links(uint8_t *self, int X, int Y, int Z, float vs, const float *origin,
                                const float *pts, const uint8_t *link_of, int64_t n, const LinkPose &poses,
                                uint32_t mask, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    Origin o{{origin[0], origin[1], origin[2]}};
    const int64_t want = (n + 255) / 256;
    const int64_t cap = static_cast<int64_t>(sm_count()) * 16;
    const int blocks = static_cast<int>(want < cap ? want : cap);
    return launch_pdl(k_insert_links, dim3(blocks), dim3(256), 0, s, self, X, Y, Z, vs, o, pts, link_of, n, poses,
                      mask);
}

cudaError_t launch_query(const QueryGrid *g, int ng, int X, int Y, int Z, float vs, const float *origin,
                         const float *centres, const float *radii, int m, vedt_sphere_result *out,
                         cudaStream_t s) {
    if (m <= 0 || ng <= 0) return cudaSuccess;
    Origin o{{origin[0], origin[1], origin[2]}};
    const int n = m * ng;
    return launch_pdl(k_query, dim3((n + 127) / 128), dim3(128), 0, s, g, ng, X, Y, Z, vs, o, centres, radii, m,
                      out);
}

}  // namespace vedt
