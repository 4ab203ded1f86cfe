// C ABI of libvedt: map lifecycle, per-frame calls, forward kinematics, timing.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "vedt_internal.h"

namespace {

// Optional NVTX ranges around the API's stages (VEDT_NVTX=1 in the environment), for
// profilers that filter launches by range (ncu --nvtx --nvtx-include ...).  Host-side
// annotations of the enqueue only; off by default.
bool nvtx_on() {
    static const bool on = [] {
        const char *e = std::getenv("VEDT_NVTX");
        return e != nullptr && e[0] == '1';
    }();
    return on;
}

struct NvtxRange {
    bool on;
    explicit NvtxRange(const char *name) : on(nvtx_on()) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxRange() {
        if (on) nvtxRangePop();
    }
};

}  // namespace

using namespace vedt;

namespace {

vedt_status from_cuda(cudaError_t e) { return e == cudaSuccess ? VEDT_OK : (e == cudaErrorMemoryAllocation ? VEDT_ENOMEM : VEDT_ECUDA); }

#define VCHECK(call)                                  \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return from_cuda(e_);  \
    } while (0)

cudaEvent_t take_event(vedt_map *m) {
    if (!m->free_events.empty()) {
        cudaEvent_t e = m->free_events.back();
        m->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records an event before a launch when timing is on; returns the pending slot or -1.
int timing_begin(vedt_map *m, int kind) {
    if (!m->timing) return -1;
    EvPair p{kind, take_event(m), take_event(m)};
    cudaEventRecord(p.a, m->stream);
    m->pending.push_back(p);
    return static_cast<int>(m->pending.size()) - 1;
}

void timing_end(vedt_map *m, int slot) {
    if (slot >= 0) cudaEventRecord(m->pending[slot].b, m->stream);
}

void harvest(vedt_map *m) {
    for (auto &p : m->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
            m->ms[p.kind] += t;
            m->cnt[p.kind] += 1;
        }
        m->free_events.push_back(p.a);
        m->free_events.push_back(p.b);
    }
    m->pending.clear();
}

bool valid_which(int w) { return w == VEDT_MAP_ENV || w == VEDT_MAP_SELF || w == VEDT_MAP_BOTH; }

}  // namespace

namespace vedt {

CUresult encode_tmap(CUtensorMap *m, CUtensorMapDataType t, int elem, void *base, uint64_t d0, uint64_t d1,
                     uint64_t d2, uint32_t b0, uint32_t b1, uint32_t b2) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    if (!fn) return CUDA_ERROR_NOT_FOUND;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * elem, d0 * d1 * elem};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, t, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

int default_pzx(const GridDesc *grids, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (grids[i].X % 8 != 0) return 32;
    return 8;
}

// Fills desc/tmaps for grids (host copies) and uploads them; used by maps and batches.
// pzx: pass-Z tile width of a small table (8 or 32; 0: default_pzx).
vedt_status build_table(GridTable &t, const std::vector<GridDesc> &grids, void *dev_desc, void *dev_tmaps,
                        int32_t *err, int pzx) {
    std::vector<GridDesc> d(grids);
    std::vector<CUtensorMap> tm(2 * grids.size());
    int64_t rows = 0, ty = 0, tz = 0;
    t.large = 0;
    t.maxY = t.maxZ = t.maxXp = 0;
    for (const GridDesc &g : d) t.large |= g.X > kSmallMax || g.Y > kSmallMax || g.Z > kSmallMax;
    const bool big = t.large != 0;
    t.pzx = pzx ? pzx : default_pzx(d.data(), d.size());
    const int px = t.pzx, py = kEnvCols / px;
    for (size_t i = 0; i < d.size(); ++i) {
        GridDesc &g = d[i];
        g.row_begin = rows;
        g.ty_begin = ty;
        g.tz_begin = tz;
        rows += static_cast<int64_t>(g.Y) * g.Z;
        ty += static_cast<int64_t>(g.Xp / kEnvCols) * g.Z;
        tz += small_tiles_z(g.Xp, g.Y, px);
        t.maxY = g.Y > t.maxY ? g.Y : t.maxY;
        t.maxZ = g.Z > t.maxZ ? g.Z : t.maxZ;
        t.maxXp = g.Xp > t.maxXp ? g.Xp : t.maxXp;
    }
    for (size_t i = 0; i < d.size(); ++i) {
        GridDesc &g = d[i];
        const uint32_t by = g.Y > kBox ? kBox : g.Y, bz = g.Z > kBox ? kBox : g.Z;
        if (encode_tmap(&tm[2 * i], big ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                        big ? 2 : 1, g.xs, g.Xp, g.Y, g.Z, kEnvCols, by, 1) != CUDA_SUCCESS)
            return VEDT_ECUDA;
        // a px x py patch of columns (rows y >= Y of a ragged last patch read as zeros)
        const CUresult r = encode_tmap(&tm[2 * i + 1], big ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                                       big ? 4 : 2, g.s2, g.Xp, g.Y, g.Z, static_cast<uint32_t>(px),
                                       static_cast<uint32_t>(py), bz);
        if (r != CUDA_SUCCESS) return VEDT_ECUDA;
    }
    VCHECK(cudaMemcpy(dev_desc, d.data(), sizeof(GridDesc) * d.size(), cudaMemcpyHostToDevice));
    VCHECK(cudaMemcpy(dev_tmaps, tm.data(), sizeof(CUtensorMap) * tm.size(), cudaMemcpyHostToDevice));
    t.desc = static_cast<GridDesc *>(dev_desc);
    t.tmaps = static_cast<CUtensorMap *>(dev_tmaps);
    t.n = static_cast<int>(d.size());
    t.rows = rows;
    t.tiles_y = ty;
    t.tiles_z = tz;
    t.err = err;
    return VEDT_OK;
}

}  // namespace vedt

namespace {

void free_map(vedt_map *m) {
    for (int i = 0; i < 2; ++i) {
        if (i == 0) {
            cudaFree(m->occ[0]);   // both grids share one allocation
            cudaFree(m->snap);
            cudaFree(m->changed);
            cudaFree(m->logodds);
        }
        cudaFree(m->sq[i]);
        cudaFree(m->ix[i]);
        cudaFree(m->xs[i]);
        cudaFree(m->row_has[i]);
        cudaFree(m->s2[i]);
        cudaFree(m->slice_has[i]);
    }
    cudaFree(m->err);
    cudaFree(m->tab_mem);
    cudaFree(m->qgrids);
    cudaFree(m->q_in);
    cudaFree(m->q_out);
    cudaFree(m->link_pts);
    cudaFree(m->link_of);
    for (int b = 0; b < 2; ++b) {
        cudaFree(m->stage[b]);
        if (m->copied[b]) cudaEventDestroy(m->copied[b]);
    }
    for (int s = 0; s < kQRing; ++s)
        if (m->fdone[s]) cudaEventDestroy(m->fdone[s]);
    if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
    if (m->pin_q) cudaFreeHost(m->pin_q);
    if (m->side_stream) cudaStreamDestroy(m->side_stream);
    if (m->links_done) cudaEventDestroy(m->links_done);
    if (m->self_done) cudaEventDestroy(m->self_done);
    if (m->done) cudaEventDestroy(m->done);
    for (auto &p : m->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : m->free_events) cudaEventDestroy(e);
    delete m;
}

GridDesc grid_of(const vedt_map *m, int i) {
    GridDesc g{};
    g.occ = m->occ[i];
    g.xs = m->xs[i];
    g.row_has = m->row_has[i];
    g.s2 = m->s2[i];
    g.slice_has = m->slice_has[i];
    g.sqdist = m->sq[i];
    g.idx = m->ix[i];
    g.X = m->X;
    g.Y = m->Y;
    g.Z = m->Z;
    g.Xp = m->Xp;
    g.changed = m->changed + i;
    return g;
}

// The map's three EDT tables, ENV = {0}, SELF = {1}, BOTH = {0, 1}, in tab_mem: four
// descriptors, then the tensor maps (128-byte aligned).  pzx: pass-Z tile width (0:
// default).  Keeps the tables' band counts.
vedt_status build_map_tables(vedt_map *m, int pzx) {
    char *base = static_cast<char *>(m->tab_mem);
    char *tmb = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(base + sizeof(GridDesc) * 4) + 127) &
                                         ~uintptr_t(127));
    const std::vector<GridDesc> g0{grid_of(m, 0)}, g1{grid_of(m, 1)}, g01{grid_of(m, 0), grid_of(m, 1)};
    vedt_status st = build_table(m->tab[0], g0, base, tmb, m->err, pzx);
    if (st == VEDT_OK)
        st = build_table(m->tab[1], g1, base + sizeof(GridDesc), tmb + 2 * sizeof(CUtensorMap), m->err, pzx);
    if (st == VEDT_OK)
        st = build_table(m->tab[2], g01, base + 2 * sizeof(GridDesc), tmb + 4 * sizeof(CUtensorMap), m->err, pzx);
    return st;
}

}  // namespace

extern "C" {

const char *vedt_version(void) {
#ifdef VEDT_DEBUG_BOUNDS
    return "vedt 0.1 (sm_103a, index checks)";
#else
    return "vedt 0.1 (sm_103a)";
#endif
}

const char *vedt_status_string(vedt_status s) {
    switch (s) {
        case VEDT_OK: return "ok";
        case VEDT_EINVAL: return "invalid argument";
        case VEDT_ENOMEM: return "out of memory";
        case VEDT_ECUDA: return "CUDA error";
        case VEDT_ETIMEOUT: return "in-kernel wait timed out";
        case VEDT_EBUSY: return "not enough free device memory";
        case VEDT_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

vedt_status vedt_map_create(const int32_t dims[3], float voxel_size, const float origin[3], void *stream,
                            vedt_map **out) {
    if (!dims || !origin || !out) return VEDT_EINVAL;
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > VEDT_MAX_DIM || !std::isfinite(origin[a])) return VEDT_EINVAL;
    if (!(voxel_size > 0.f) || !std::isfinite(voxel_size)) return VEDT_EINVAL;
    vedt_map *m = new (std::nothrow) vedt_map();
    if (!m) return VEDT_ENOMEM;
    m->X = dims[0];
    m->Y = dims[1];
    m->Z = dims[2];
    m->Xp = (m->X + kTile - 1) / kTile * kTile;
    m->vs = voxel_size;
    for (int a = 0; a < 3; ++a) m->origin[a] = origin[a];
    m->stream = static_cast<cudaStream_t>(stream);
    m->large = (m->X > kSmallMax || m->Y > kSmallMax || m->Z > kSmallMax) ? 1 : 0;
    m->N = static_cast<int64_t>(m->X) * m->Y * m->Z;
    const int64_t Np = static_cast<int64_t>(m->Xp) * m->Y * m->Z;
    const size_t s2b = m->large ? 4 : 2;
    cudaError_t e = cudaSuccess;
    // both occupancy grids in one allocation, M_S 256-byte aligned right after M_I, so a
    // frame's ClearMap of both is a single launch
    const int64_t n_al = (m->N + 255) / 256 * 256;
    e = cudaMalloc(&m->occ[0], 2 * n_al);
    if (e == cudaSuccess) m->occ[1] = m->occ[0] + n_al;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (e == cudaSuccess) e = cudaMalloc(&m->sq[i], m->N * 4);
        if (e == cudaSuccess) e = cudaMalloc(&m->ix[i], m->N * 4);
        if (e == cudaSuccess) e = cudaMalloc(&m->xs[i], Np * (m->large ? 2 : 1));
        if (e == cudaSuccess) e = cudaMalloc(&m->row_has[i], static_cast<int64_t>(m->Y) * m->Z);
        if (e == cudaSuccess) e = cudaMalloc(&m->s2[i], Np * s2b);
        if (e == cudaSuccess) e = cudaMalloc(&m->slice_has[i], m->Z);
    }
    if (e == cudaSuccess) e = cudaMalloc(&m->err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&m->changed, 2 * sizeof(uint32_t));
    const size_t desc_bytes = sizeof(GridDesc) * 4, tm_bytes = sizeof(CUtensorMap) * 8;
    if (e == cudaSuccess) e = cudaMalloc(&m->tab_mem, desc_bytes + tm_bytes + 256);
    if (e == cudaSuccess) e = cudaMalloc(&m->qgrids, sizeof(QueryGrid) * 4);
    // query input area of vedt_query_spheres (host frames read page-locked slots in place)
    if (e == cudaSuccess) e = cudaMalloc(&m->q_in, sizeof(float) * 4 * kMaxQuery);
    if (e == cudaSuccess) e = cudaMalloc(&m->q_out, sizeof(vedt_sphere_result) * 2 * kMaxQuery);
    if (e != cudaSuccess) {
        free_map(m);
        return from_cuda(e);
    }
    e = cudaMemset(m->err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(m->changed, 1, 2 * sizeof(uint32_t));   // nonzero: recompute
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMemset(m->occ[i], 0, m->N);
    if (e != cudaSuccess) {
        free_map(m);
        return from_cuda(e);
    }
    vedt_status st = build_map_tables(m, 0);
    const QueryGrid qg[4] = {{m->sq[0], m->ix[0]}, {m->sq[1], m->ix[1]}, {m->sq[0], m->ix[0]}, {m->sq[1], m->ix[1]}};
    if (st == VEDT_OK) st = from_cuda(cudaMemcpy(m->qgrids, qg, sizeof(qg), cudaMemcpyHostToDevice));
    if (st != VEDT_OK) {
        free_map(m);
        return st;
    }
    *out = m;
    return VEDT_OK;
}

vedt_status vedt_map_destroy(vedt_map *m) {
    if (!m) return VEDT_OK;
    cudaStreamSynchronize(m->stream);
    for (cudaStream_t x : {m->side_stream, m->copy_stream})
        if (x) cudaStreamSynchronize(x);
    free_map(m);
    return VEDT_OK;
}

vedt_status vedt_map_set_stream(vedt_map *m, void *stream) {
    if (!m) return VEDT_EINVAL;
    m->stream = static_cast<cudaStream_t>(stream);
    return VEDT_OK;
}

vedt_status vedt_map_set_logodds(vedt_map *m, int on, int l_hit, int l_miss, int l_min, int l_max,
                                 int threshold) {
    if (!m) return VEDT_EINVAL;
    if (on && (l_hit < 0 || l_hit > 255 || l_miss < 0 || l_miss > 255 || l_min < -128 || l_min > 0 ||
               l_max < 0 || l_max > 127 || threshold <= l_min))
        return VEDT_EINVAL;
    VCHECK(cudaStreamSynchronize(m->stream));
    if (m->side_stream) VCHECK(cudaStreamSynchronize(m->side_stream));
    cudaFree(m->logodds);
    m->logodds = nullptr;
    if (!on) return VEDT_OK;
    const int64_t n_al = m->occ[1] - m->occ[0];
    cudaError_t e = cudaMalloc(&m->logodds, n_al);
    if (e == cudaSuccess) e = cudaMemset(m->logodds, 0, n_al);   // 0: unknown
    if (e != cudaSuccess) {
        cudaFree(m->logodds);
        m->logodds = nullptr;
        return from_cuda(e);
    }
    const int p[5] = {l_hit, l_miss, l_min, l_max, threshold};
    for (int k = 0; k < 5; ++k) m->lo_param[k] = p[k];
    return VEDT_OK;
}

vedt_status vedt_update_occupancy(vedt_map *m) {
    const NvtxRange nvtx_range("vedt_update_occupancy");
    if (!m || !m->logodds) return VEDT_EINVAL;
    const int slot = timing_begin(m, VEDT_K_OCCUPANCY);
    VCHECK(launch_logodds(m->occ[0], m->logodds, m->N, m->lo_param, m->stream));
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_map_set_incremental(vedt_map *m, int on) {
    if (!m) return VEDT_EINVAL;
    VCHECK(cudaStreamSynchronize(m->stream));
    const int64_t n_al = m->occ[1] - m->occ[0];
    if (on && !m->snap) {
        const cudaError_t e = cudaMalloc(&m->snap, 2 * n_al);
        if (e != cudaSuccess) {
            m->snap = nullptr;
            return from_cuda(e);
        }
    }
    if (!on && m->snap) {
        cudaFree(m->snap);
        m->snap = nullptr;
    }
    m->incremental = on ? 1 : 0;
    m->snap_valid[0] = m->snap_valid[1] = false;   // the first EDT after a switch recomputes
    for (GridTable &t : m->tab) t.incr = m->incremental;
    VCHECK(cudaMemset(m->changed, 1, 2 * sizeof(uint32_t)));
    return VEDT_OK;
}

vedt_status vedt_map_edt_recomputed(vedt_map *m, int which, int32_t *out) {
    if (!m || !out || !valid_which(which)) return VEDT_EINVAL;
    VCHECK(cudaStreamSynchronize(m->stream));
    uint32_t c[2] = {1, 1};
    VCHECK(cudaMemcpy(c, m->changed, sizeof(c), cudaMemcpyDeviceToHost));
    int k = 0;
    if (which & VEDT_MAP_ENV) out[k++] = c[0] != 0;
    if (which & VEDT_MAP_SELF) out[k++] = c[1] != 0;
    return VEDT_OK;
}

vedt_status vedt_map_set_bands(vedt_map *m, int bands) {
    if (!m) return VEDT_EINVAL;
    const bool large = m->tab[0].large != 0;
    const bool ok = bands == 0 || bands == 4 || bands == 8 || (!large && (bands == 1 || bands == 2));
    if (!ok) return VEDT_EINVAL;
    for (GridTable &t : m->tab) t.bands = bands;
    return VEDT_OK;
}

vedt_status vedt_map_set_tile_z(vedt_map *m, int cols_x) {
    if (!m || !(cols_x == 0 || cols_x == 8 || cols_x == 32)) return VEDT_EINVAL;
    // the tables' device descriptors and tensor maps are rewritten: nothing of this map
    // may be in flight
    VCHECK(cudaStreamSynchronize(m->stream));
    if (m->side_stream) VCHECK(cudaStreamSynchronize(m->side_stream));
    if (m->copy_stream) VCHECK(cudaStreamSynchronize(m->copy_stream));
    return build_map_tables(m, cols_x);
}

int vedt_map_tile_z(const vedt_map *m) { return m ? m->tab[0].pzx : 0; }

vedt_status vedt_map_info(const vedt_map *m, int32_t dims_out[3], float *vs, float origin_out[3]) {
    if (!m) return VEDT_EINVAL;
    if (dims_out) {
        dims_out[0] = m->X;
        dims_out[1] = m->Y;
        dims_out[2] = m->Z;
    }
    if (vs) *vs = m->vs;
    if (origin_out)
        for (int a = 0; a < 3; ++a) origin_out[a] = m->origin[a];
    return VEDT_OK;
}

vedt_status vedt_clear(vedt_map *m, int which) {
    const NvtxRange nvtx_range("vedt_clear");
    if (!m || !valid_which(which)) return VEDT_EINVAL;
    const int slot = timing_begin(m, VEDT_K_CLEAR);
    if (which == VEDT_MAP_BOTH) {
        VCHECK(launch_clear(m->occ[0], m->occ[1] - m->occ[0] + m->N, m->stream));
    } else {
        VCHECK(launch_clear(m->occ[which == VEDT_MAP_ENV ? 0 : 1], m->N, m->stream));
    }
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_insert_pointcloud_masked(vedt_map *m, const float *xyz_dev, int64_t n, const float *T,
                                          int filter_self, const uint8_t *keep_dev, int64_t *counts_dev) {
    const NvtxRange nvtx_range("vedt_insert_pointcloud");
    if (!m || n < 0 || (n > 0 && !xyz_dev)) return VEDT_EINVAL;
    if (n == 0) return VEDT_OK;
    const int slot = timing_begin(m, VEDT_K_INSERT_POINTS);
    VCHECK(launch_insert_points(m->occ[0], m->occ[1], m->X, m->Y, m->Z, m->vs, m->origin, xyz_dev, n, T,
                                filter_self ? 1 : 0, keep_dev, counts_dev, m->stream));
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_insert_pointcloud(vedt_map *m, const float *xyz_dev, int64_t n, const float *T,
                                   int filter_self, int64_t *counts_dev) {
    return vedt_insert_pointcloud_masked(m, xyz_dev, n, T, filter_self, nullptr, counts_dev);
}

vedt_status vedt_register_links(vedt_map *m, int n_links, const float *const *xyz, const int64_t *n_vox) {
    if (!m || n_links < 1 || n_links > VEDT_MAX_LINKS || !xyz || !n_vox) return VEDT_EINVAL;
    int64_t total = 0;
    for (int k = 0; k < n_links; ++k) {
        if (n_vox[k] < 0 || (n_vox[k] > 0 && !xyz[k])) return VEDT_EINVAL;
        total += n_vox[k];
    }
    std::vector<float> pts(static_cast<size_t>(total) * 3);
    std::vector<uint8_t> of(static_cast<size_t>(total));
    int64_t w = 0;
    for (int k = 0; k < n_links; ++k) {
        if (n_vox[k] > 0) std::memcpy(pts.data() + 3 * w, xyz[k], sizeof(float) * 3 * n_vox[k]);
        std::memset(of.data() + w, k, static_cast<size_t>(n_vox[k]));
        w += n_vox[k];
    }
    VCHECK(cudaStreamSynchronize(m->stream));
    cudaFree(m->link_pts);
    cudaFree(m->link_of);
    m->link_pts = nullptr;
    m->link_of = nullptr;
    m->n_link_pts = 0;
    m->n_links = 0;
    if (total > 0) {
        VCHECK(cudaMalloc(&m->link_pts, pts.size() * sizeof(float)));
        VCHECK(cudaMalloc(&m->link_of, of.size()));
        VCHECK(cudaMemcpy(m->link_pts, pts.data(), pts.size() * sizeof(float), cudaMemcpyHostToDevice));
        VCHECK(cudaMemcpy(m->link_of, of.data(), of.size(), cudaMemcpyHostToDevice));
    }
    m->n_link_pts = total;
    m->n_links = n_links;
    return VEDT_OK;
}

vedt_status vedt_insert_links(vedt_map *m, const float *poses, uint32_t mask) {
    const NvtxRange nvtx_range("vedt_insert_links");
    if (!m || !poses || m->n_links == 0) return VEDT_EINVAL;
    if (m->n_links < 32 && (mask >> m->n_links) != 0u) return VEDT_EINVAL;
    LinkPose P{};
    for (int k = 0; k < m->n_links; ++k)
        for (int i = 0; i < 12; ++i) P.T[k][i] = poses[12 * k + i];
    const int slot = timing_begin(m, VEDT_K_INSERT_LINKS);
    VCHECK(launch_insert_links(m->occ[1], m->X, m->Y, m->Z, m->vs, m->origin, m->link_pts, m->link_of,
                               m->n_link_pts, P, mask, m->stream));
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_fk(const vedt_chain *c, const double *q, double *out) {
    if (!c || !q || !out || c->n_joints < 1 || c->n_joints > VEDT_MAX_JOINTS) return VEDT_EINVAL;
    // T_0 = base; T_k = T_(k-1) * offset_k * Rz(q_k); every entry summed left to right.
    auto mul = [](const double *A, const double *B, double *C) {
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                double s = A[4 * i] * B[j];
                s = s + A[4 * i + 1] * B[4 + j];
                s = s + A[4 * i + 2] * B[8 + j];
                C[4 * i + j] = s;
            }
            double t = A[4 * i] * B[3];
            t = t + A[4 * i + 1] * B[7];
            t = t + A[4 * i + 2] * B[11];
            C[4 * i + 3] = t + A[4 * i + 3];
        }
    };
    std::memcpy(out, c->base, sizeof(double) * 12);
    for (int k = 0; k < c->n_joints; ++k) {
        const double cq = std::cos(q[k]), sq = std::sin(q[k]);
        const double rz[12] = {cq, -sq, 0.0, 0.0, sq, cq, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0};
        double tmp[12];
        mul(out + 12 * k, c->offset[k], tmp);
        mul(tmp, rz, out + 12 * (k + 1));
    }
    return VEDT_OK;
}

vedt_status vedt_fk_batch(const vedt_chain *c, const double *q, int64_t n, double *poses_out) {
    if (!c || (n > 0 && (!q || !poses_out)) || n < 0) return VEDT_EINVAL;
    const int J = c->n_joints;
    for (int64_t i = 0; i < n; ++i) {
        const vedt_status st = vedt_fk(c, q + i * J, poses_out + i * (J + 1) * 12);
        if (st != VEDT_OK) return st;
    }
    return VEDT_OK;
}

vedt_status vedt_sphere_centres(const vedt_chain *c, const double *q, int n, const int32_t *link_of,
                                const double *local, float *out) {
    if (!c || n < 0 || c->n_joints < 1 || c->n_joints > VEDT_MAX_JOINTS) return VEDT_EINVAL;
    if (n == 0) return VEDT_OK;
    if (!q || !link_of || !local || !out) return VEDT_EINVAL;
    for (int i = 0; i < n; ++i)
        if (link_of[i] < 0 || link_of[i] > c->n_joints) return VEDT_EINVAL;
    double P[(VEDT_MAX_JOINTS + 1) * 12];
    const vedt_status st = vedt_fk(c, q, P);
    if (st != VEDT_OK) return st;
    for (int i = 0; i < n; ++i) {
        const double *T = P + 12 * link_of[i];
        const double *l = local + 3 * i;
        for (int a = 0; a < 3; ++a) {
            double s = T[4 * a] * l[0];
            s = s + T[4 * a + 1] * l[1];
            s = s + T[4 * a + 2] * l[2];
            out[3 * i + a] = static_cast<float>(s + T[4 * a + 3]);
        }
    }
    return VEDT_OK;
}

vedt_status vedt_sphere_centres_batch(const vedt_chain *c, const double *q, int64_t n, int m, const int32_t *link_of,
                                      const double *local, float *out) {
    if (!c || n < 0 || m < 0 || c->n_joints < 1 || c->n_joints > VEDT_MAX_JOINTS) return VEDT_EINVAL;
    if (n == 0 || m == 0) return VEDT_OK;
    if (!q) return VEDT_EINVAL;
    for (int64_t k = 0; k < n; ++k) {
        const vedt_status st = vedt_sphere_centres(c, q + k * c->n_joints, m, link_of, local, out + k * m * 3);
        if (st != VEDT_OK) return st;
    }
    return VEDT_OK;
}

vedt_status vedt_insert_robot(vedt_map *m, const vedt_chain *c, const double *q, uint32_t mask) {
    if (!m || !c || !q || c->n_joints < 1 || c->n_joints > VEDT_MAX_JOINTS) return VEDT_EINVAL;
    if (c->n_joints + 1 > m->n_links) return VEDT_EINVAL;
    double P[(VEDT_MAX_JOINTS + 1) * 12];
    vedt_status st = vedt_fk(c, q, P);
    if (st != VEDT_OK) return st;
    float Pf[VEDT_MAX_LINKS * 12] = {};
    for (int i = 0; i < (c->n_joints + 1) * 12 && i < VEDT_MAX_LINKS * 12; ++i) Pf[i] = static_cast<float>(P[i]);
    return vedt_insert_links(m, Pf, mask);
}

vedt_status vedt_compute_edt(vedt_map *m, int which) {
    const NvtxRange nvtx_range("vedt_compute_edt");
    if (!m || !valid_which(which)) return VEDT_EINVAL;
    const GridTable &t = m->tab[which - 1];
    int slot = timing_begin(m, VEDT_K_EDT_X);
    if (m->incremental) {
        // per grid: changed = 0, then the diff kernel sets it if the occupancy differs from
        // the snapshot of the last EDT; a grid whose fields are not known to match its
        // snapshot is recomputed regardless
        const int g0 = which == VEDT_MAP_SELF ? 1 : 0, ng = which == VEDT_MAP_BOTH ? 2 : 1;
        const int64_t n_al = m->occ[1] - m->occ[0];
        for (int g = g0; g < g0 + ng; ++g)
            VCHECK(cudaMemsetAsync(m->changed + g, m->snap_valid[g] ? 0 : 1, sizeof(uint32_t), m->stream));
        VCHECK(launch_occ_diff(m->occ[g0], m->snap + g0 * n_al, m->changed + g0, n_al, ng, m->stream));
        for (int g = g0; g < g0 + ng; ++g) m->snap_valid[g] = true;
    }
    VCHECK(launch_pass_x(t, m->stream, (m->fuse_lo && which == VEDT_MAP_ENV) ? m->logodds : nullptr, m->lo_param));
    timing_end(m, slot);
    slot = timing_begin(m, VEDT_K_EDT_Y);
    VCHECK(launch_pass_y(t, m->stream));
    timing_end(m, slot);
    slot = timing_begin(m, VEDT_K_EDT_Z);
    VCHECK(launch_pass_z(t, m->stream));
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_query_spheres_dev(vedt_map *m, const float *centres, const float *radii, int n, int which,
                                   vedt_sphere_result *out) {
    const NvtxRange nvtx_range("vedt_query_spheres");
    if (!m || !centres || !radii || !out || n < 1 || n > kMaxQuery || !valid_which(which)) return VEDT_EINVAL;
    const QueryGrid *g = which == VEDT_MAP_SELF ? m->qgrids + 1 : m->qgrids;
    const int ng = which == VEDT_MAP_BOTH ? 2 : 1;
    const int slot = timing_begin(m, VEDT_K_QUERY);
    VCHECK(launch_query(g, ng, m->X, m->Y, m->Z, m->vs, m->origin, centres, radii, n, out, m->stream));
    timing_end(m, slot);
    return VEDT_OK;
}

vedt_status vedt_check(vedt_map *m) {
    if (!m) return VEDT_EINVAL;
    VCHECK(cudaStreamSynchronize(m->stream));
    int32_t e = 0;
    VCHECK(cudaMemcpy(&e, m->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) {
        VCHECK(cudaMemset(m->err, 0, sizeof(int32_t)));
        return (e & kErrTimeout) ? VEDT_ETIMEOUT : VEDT_ECUDA;
    }
    return VEDT_OK;
}

vedt_status vedt_query_spheres(vedt_map *m, const float *centres, const float *radii, int n, int which,
                               vedt_sphere_result *out) {
    if (!m || !centres || !radii || !out || n < 1 || n > kMaxQuery || !valid_which(which)) return VEDT_EINVAL;
    VCHECK(cudaMemcpyAsync(m->q_in, centres, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m->stream));
    VCHECK(cudaMemcpyAsync(m->q_in + 3 * kMaxQuery, radii, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
    vedt_status st = vedt_query_spheres_dev(m, m->q_in, m->q_in + 3 * kMaxQuery, n, which, m->q_out);
    if (st != VEDT_OK) return st;
    const int ng = which == VEDT_MAP_BOTH ? 2 : 1;
    VCHECK(cudaMemcpyAsync(out, m->q_out, sizeof(vedt_sphere_result) * n * ng, cudaMemcpyDeviceToHost, m->stream));
    return vedt_check(m);
}

vedt_status vedt_frame(vedt_map *m, const float *xyz, int64_t n, const float *T, const vedt_chain *chain,
                       const double *q, uint32_t mask, const float *centres, const float *radii, int nq,
                       vedt_sphere_result *out) {
    const NvtxRange nvtx_range("vedt_frame");
    if (!m || n < 0 || (n > 0 && !xyz) || (chain && !q) || nq < 0 || nq > kMaxQuery) return VEDT_EINVAL;
    if (nq > 0 && (!centres || !radii || !out)) return VEDT_EINVAL;
    vedt_status st = vedt_clear(m, VEDT_MAP_BOTH);
    if (st == VEDT_OK && chain) st = vedt_insert_robot(m, chain, q, mask);
    if (st != VEDT_OK) return st;
    if (m->timing) {
        // per-kernel timing: the same launches, one after another on the map's stream, so
        // that each launch's events time that kernel alone
        st = vedt_compute_edt(m, VEDT_MAP_SELF);
        if (st == VEDT_OK) st = vedt_insert_pointcloud(m, xyz, n, T, 1, nullptr);
        if (st == VEDT_OK && m->logodds) st = vedt_update_occupancy(m);
        if (st == VEDT_OK) st = vedt_compute_edt(m, VEDT_MAP_ENV);
        if (st == VEDT_OK && nq > 0) st = vedt_query_spheres_dev(m, centres, radii, nq, VEDT_MAP_BOTH, out);
        return st;
    }
    if (!m->side_stream) {   // created together, or not at all
        cudaStream_t side = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (b) cudaEventDestroy(b);
            if (a) cudaEventDestroy(a);
            if (side) cudaStreamDestroy(side);
            return from_cuda(e);
        }
        m->side_stream = side;
        m->links_done = a;
        m->self_done = b;
    }
    // M_S is final once the links are in: its EDT overlaps the point insertion and M_I's EDT
    VCHECK(cudaEventRecord(m->links_done, m->stream));
    VCHECK(cudaStreamWaitEvent(m->side_stream, m->links_done, 0));
    cudaStream_t main = m->stream;
    m->stream = m->side_stream;
    st = vedt_compute_edt(m, VEDT_MAP_SELF);
    m->stream = main;
    if (st != VEDT_OK) return st;
    VCHECK(cudaEventRecord(m->self_done, m->side_stream));
    st = vedt_insert_pointcloud(m, xyz, n, T, 1, nullptr);
    // the log-odds update rides in M_I's pass X (small grids, no incremental snapshot,
    // which must see the updated occupancy before pass X); else its own kernel
    const bool fuse = m->logodds && !m->incremental && !m->tab[VEDT_MAP_ENV - 1].large;
    if (st == VEDT_OK && m->logodds && !fuse) st = vedt_update_occupancy(m);
    if (st == VEDT_OK) {
        m->fuse_lo = fuse;
        st = vedt_compute_edt(m, VEDT_MAP_ENV);
        m->fuse_lo = false;
    }
    if (st != VEDT_OK) return st;
    VCHECK(cudaStreamWaitEvent(m->stream, m->self_done, 0));
    if (nq > 0) st = vedt_query_spheres_dev(m, centres, radii, nq, VEDT_MAP_BOTH, out);
    return st;
}

namespace {

// Queues one cycle from host buffers on the map's stream.  The cloud goes to staging
// buffer h % 2 on the copy stream once the frame that last read that buffer (h - 2) has
// finished, so the upload overlaps the previous frame's kernels, and the map's stream
// waits for it before the frame's kernels; the sphere centres and radii go to page-locked
// slot h % kQRing, which the frame's query reads in place.
vedt_status queue_host_frame(vedt_map *m, const float *xyz, int64_t n, const float *T, const vedt_chain *chain,
                             const double *q, uint32_t mask, const float *centres, const float *radii, int nq,
                             vedt_sphere_result *out) {
    if (!m->copy_stream) {   // created together, or not at all
        constexpr int kEv = 2 + kQRing;
        cudaStream_t cs = nullptr;
        cudaEvent_t ev[kEv] = {};
        float *pin = nullptr;
        void *pin_dev = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int j = 0; j < kEv && e == cudaSuccess; ++j) e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void **>(&pin), sizeof(float) * kQRing * 4 * kMaxQuery, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&pin_dev, pin, 0);
        if (e != cudaSuccess) {
            if (pin) cudaFreeHost(pin);
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            if (cs) cudaStreamDestroy(cs);
            return from_cuda(e);
        }
        m->copy_stream = cs;
        m->pin_q = pin;
        m->pin_q_dev = static_cast<const float *>(pin_dev);
        for (int b = 0; b < 2; ++b) m->copied[b] = ev[b];
        for (int r = 0; r < kQRing; ++r) m->fdone[r] = ev[2 + r];
    }
    if (n > m->stage_cap) {
        // Grow both buffers without synchronising the device (cudaFree would wait for every
        // stream, other maps' frames included): the old buffers are released on the map's
        // stream after the queued frames that read them, the new ones come from the
        // stream-ordered allocator on the copy stream, ahead of the uploads into them.
        for (int b = 0; b < 2; ++b) {
            if (m->stage[b]) VCHECK(cudaFreeAsync(m->stage[b], m->stream));
            m->stage[b] = nullptr;
        }
        m->stage_cap = 0;
        for (int b = 0; b < 2; ++b)
            VCHECK(cudaMallocAsync(reinterpret_cast<void **>(&m->stage[b]), sizeof(float) * 3 * n, m->copy_stream));
        m->stage_cap = n;
    }
    const int64_t h = m->hframes++;
    const int b = static_cast<int>(h & 1), r = static_cast<int>(h % kQRing);
    // the upload goes on the copy stream (the map's stream then has an event wait between
    // frames instead of a copy, which would end the programmatic overlap of one frame's
    // last kernel with the next frame's first); fdone[x] holds its latest record, the end
    // of the last frame queued in slot x
    if (n > 0) {
        if (h >= 2) VCHECK(cudaStreamWaitEvent(m->copy_stream, m->fdone[(h - 2) % kQRing], 0));
        VCHECK(cudaMemcpyAsync(m->stage[b], xyz, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, m->copy_stream));
        VCHECK(cudaEventRecord(m->copied[b], m->copy_stream));
        VCHECK(cudaStreamWaitEvent(m->stream, m->copied[b], 0));
    }
    const float *qin = m->pin_q_dev + static_cast<size_t>(r) * 4 * kMaxQuery;
    if (nq > 0) {
        // slot r was last read by the query of the frame kQRing back: wait for it on the
        // host (at once unless the caller runs kQRing frames ahead of the device)
        if (h >= kQRing) VCHECK(cudaEventSynchronize(m->fdone[r]));
        float *pq = m->pin_q + static_cast<size_t>(r) * 4 * kMaxQuery;
        std::memcpy(pq, centres, sizeof(float) * 3 * nq);
        std::memcpy(pq + 3 * kMaxQuery, radii, sizeof(float) * nq);
    }
    // The results go straight into the caller's buffer when it is page-locked host memory
    // the device can address: the query kernel's stores then reach the host with the
    // frame, and no copy sits on the map's stream between this frame's query and the next
    // frame's first kernel.  Other buffers get a copy after the frame.
    vedt_sphere_result *direct = nullptr;
    if (nq > 0) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, out) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer)
                direct = static_cast<vedt_sphere_result *>(pa.devicePointer);
        } else {
            (void)cudaGetLastError();   // an address the runtime does not know: copy
        }
    }
    vedt_status st =
        vedt_frame(m, m->stage[b], n, T, chain, q, mask, qin, qin + 3 * kMaxQuery, nq, direct ? direct : m->q_out);
    if (st != VEDT_OK) return st;
    VCHECK(cudaEventRecord(m->fdone[r], m->stream));
    if (nq > 0 && !direct)
        VCHECK(cudaMemcpyAsync(out, m->q_out, sizeof(vedt_sphere_result) * 2 * nq, cudaMemcpyDeviceToHost,
                               m->stream));
    return VEDT_OK;
}

}  // namespace

vedt_status vedt_frame_host(vedt_map *m, const float *xyz, int64_t n, const float *T, const vedt_chain *chain,
                            const double *q, uint32_t mask, const float *centres, const float *radii, int nq,
                            vedt_sphere_result *out) {
    if (!m || n < 0 || (n > 0 && !xyz) || nq < 0 || nq > kMaxQuery) return VEDT_EINVAL;
    if (nq > 0 && (!centres || !radii || !out)) return VEDT_EINVAL;
    const vedt_status st = queue_host_frame(m, xyz, n, T, chain, q, mask, centres, radii, nq, out);
    if (st != VEDT_OK) return st;
    return vedt_check(m);
}

vedt_status vedt_frame_host_async(vedt_map *m, const float *xyz, int64_t n, const float *T, const vedt_chain *chain,
                                  const double *q, uint32_t mask, const float *centres, const float *radii, int nq,
                                  vedt_sphere_result *out) {
    if (!m || n < 0 || (n > 0 && !xyz) || nq < 0 || nq > kMaxQuery) return VEDT_EINVAL;
    if (nq > 0 && (!centres || !radii || !out)) return VEDT_EINVAL;
    if (!m->done) VCHECK(cudaEventCreateWithFlags(&m->done, cudaEventDisableTiming));
    const vedt_status st = queue_host_frame(m, xyz, n, T, chain, q, mask, centres, radii, nq, out);
    if (st != VEDT_OK) return st;
    VCHECK(cudaEventRecord(m->done, m->stream));
    return VEDT_OK;
}

vedt_status vedt_frame_done(vedt_map *m) {
    if (!m) return VEDT_EINVAL;
    if (!m->done) return VEDT_OK;
    const cudaError_t e = cudaEventQuery(m->done);
    if (e == cudaErrorNotReady) return VEDT_EBUSY;
    if (e != cudaSuccess) return from_cuda(e);
    int32_t err = 0;
    VCHECK(cudaMemcpy(&err, m->err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        VCHECK(cudaMemset(m->err, 0, sizeof(int32_t)));
        return (err & kErrTimeout) ? VEDT_ETIMEOUT : VEDT_ECUDA;
    }
    return VEDT_OK;
}

vedt_status vedt_selftest_wait(void *stream, uint32_t limit) {
    unsigned *counter = nullptr;
    int32_t *err = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_wait_selftest(counter, limit, err, s);
    int32_t flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(flag), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(counter);
    cudaFree(err);
    if (e != cudaSuccess) return from_cuda(e);
    return (flag & kErrTimeout) ? VEDT_ETIMEOUT : VEDT_OK;
}

int64_t vedt_map_bytes(const int32_t dims[3]) {
    if (!dims) return -1;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > VEDT_MAX_DIM) return -1;
    const bool large = dims[0] > kSmallMax || dims[1] > kSmallMax || dims[2] > kSmallMax;
    const int64_t N = static_cast<int64_t>(dims[0]) * dims[1] * dims[2];
    const int64_t Np = static_cast<int64_t>((dims[0] + kTile - 1) / kTile * kTile) * dims[1] * dims[2];
    const int64_t per_grid = N * 9 + Np * (large ? 6 : 3) + static_cast<int64_t>(dims[1]) * dims[2] + dims[2];
    return 2 * per_grid + (1 << 20);
}

vedt_status vedt_device_memory(int64_t *free_bytes, int64_t *total_bytes) {
    size_t f = 0, t = 0;
    VCHECK(cudaMemGetInfo(&f, &t));
    if (free_bytes) *free_bytes = static_cast<int64_t>(f);
    if (total_bytes) *total_bytes = static_cast<int64_t>(t);
    return VEDT_OK;
}

vedt_status vedt_get_field(vedt_map *m, int which, const int32_t **sq, const int32_t **ix) {
    if (!m || (which != VEDT_MAP_ENV && which != VEDT_MAP_SELF)) return VEDT_EINVAL;
    const int i = which == VEDT_MAP_ENV ? 0 : 1;
    if (sq) *sq = m->sq[i];
    if (ix) *ix = m->ix[i];
    return VEDT_OK;
}

vedt_status vedt_get_occupancy(vedt_map *m, int which, uint8_t **occ) {
    if (!m || !occ || (which != VEDT_MAP_ENV && which != VEDT_MAP_SELF)) return VEDT_EINVAL;
    *occ = m->occ[which == VEDT_MAP_ENV ? 0 : 1];
    return VEDT_OK;
}

vedt_status vedt_set_timing(vedt_map *m, int enable) {
    if (!m) return VEDT_EINVAL;
    m->timing = enable != 0;
    return VEDT_OK;
}

vedt_status vedt_kernel_times(vedt_map *m, double *ms_out, int64_t *count_out) {
    if (!m) return VEDT_EINVAL;
    VCHECK(cudaStreamSynchronize(m->stream));
    harvest(m);
    for (int k = 0; k < VEDT_NUM_KERNELS; ++k) {
        if (ms_out) ms_out[k] = m->ms[k];
        if (count_out) count_out[k] = m->cnt[k];
        m->ms[k] = 0;
        m->cnt[k] = 0;
    }
    return VEDT_OK;
}

}  // extern "C"
