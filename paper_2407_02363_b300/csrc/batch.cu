// Batches of maps: many independent maps of uneven extents and joint states processed
// together, with the per-frame pipeline (ClearMap, Insert(O_Lk), Insert(Point_Cloud),
// PBA_EDT, ExtractClosestObstaclePose; Alg. 2 lines 4-10) as a handful of launches over
// all maps -- the EDT as one persistent launch -- optionally recorded once as a CUDA
// graph and replayed every frame.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vedt_internal.h"

using namespace vedt;

namespace {

// one member map as the batched pipeline kernels see it
struct MapRef {
    uint8_t *occ[2];
    int32_t *sq[2];
    int32_t *ix[2];
    int32_t X, Y, Z, pad;
    float vs, o[3];
    int64_t N;
};


// ClearMap of both grids of every map: blockIdx.y = map * 2 + grid.
__global__ void __launch_bounds__(256) k_clear_many(const MapRef *__restrict__ maps) {
    const MapRef &M = maps[blockIdx.y >> 1];
    uint8_t *p = M.occ[blockIdx.y & 1];
    const int64_t n = M.N;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t nvec = n >> 4;   // grids come from cudaMalloc: 256-byte aligned
    uint4 *v = reinterpret_cast<uint4 *>(p);
    for (int64_t i = tid; i < nvec; i += stride) v[i] = make_uint4(0, 0, 0, 0);
    for (int64_t i = (nvec << 4) + tid; i < n; i += stride) p[i] = 0;
}

// UpdateLinks + Insert(O_Lk) for every map: blockIdx.y = map; the link model is shared,
// each map has its own poses [map][link][12].
__global__ void __launch_bounds__(256) k_insert_links_many(const MapRef *__restrict__ maps,
                                                           const float *__restrict__ pts,
                                                           const uint8_t *__restrict__ link_of, int64_t n,
                                                           const float *__restrict__ poses, uint32_t mask) {
    const MapRef &M = maps[blockIdx.y];
    const float *P = poses + static_cast<int64_t>(blockIdx.y) * VEDT_MAX_LINKS * 12;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int k = link_of[i];
        if (!((mask >> k) & 1u)) continue;
        float wx, wy, wz;
        rigid(P + 12 * k, __ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2), wx, wy, wz);
        int vx, vy, vz;
        if (!voxel_coord(wx, M.o[0], M.vs, M.X, vx) || !voxel_coord(wy, M.o[1], M.vs, M.Y, vy) ||
            !voxel_coord(wz, M.o[2], M.vs, M.Z, vz))
            continue;
        M.occ[1][vx + static_cast<int64_t>(M.X) * (vy + static_cast<int64_t>(M.Y) * vz)] = 1;
    }
}

// Insert(Point_Cloud) with robot-point removal for every map: map m owns points
// [offs[m], offs[m+1]) of the shared world-frame buffer.
__global__ void __launch_bounds__(256) k_insert_points_many(const MapRef *__restrict__ maps,
                                                            const float *__restrict__ xyz,
                                                            const int64_t *__restrict__ offs) {
    const MapRef &M = maps[blockIdx.y];
    const int64_t b = offs[blockIdx.y], e = offs[blockIdx.y + 1];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = b + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < e; i += stride) {
        int vx, vy, vz;
        if (!voxel_coord(__ldg(xyz + 3 * i), M.o[0], M.vs, M.X, vx) ||
            !voxel_coord(__ldg(xyz + 3 * i + 1), M.o[1], M.vs, M.Y, vy) ||
            !voxel_coord(__ldg(xyz + 3 * i + 2), M.o[2], M.vs, M.Z, vz))
            continue;
        const int64_t id = vx + static_cast<int64_t>(M.X) * (vy + static_cast<int64_t>(M.Y) * vz);
        if (M.occ[1][id]) continue;
        M.occ[0][id] = 1;
    }
}

// ExtractClosestObstaclePose + Eq. (dist) for every map: thread (map, grid, sphere);
// results [map][grid][sphere], environment grid first.
__global__ void __launch_bounds__(128) k_query_many(const MapRef *__restrict__ maps, int n_maps,
                                                    const float *__restrict__ centres,
                                                    const float *__restrict__ radii, int m,
                                                    vedt_sphere_result *__restrict__ out) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(n_maps) * 2 * m) return;
    const int i = static_cast<int>(t % m);
    const int g = static_cast<int>((t / m) & 1);
    const int mi = static_cast<int>(t / (2 * m));
    const MapRef &M = maps[mi];
    const float *c = centres + (static_cast<int64_t>(mi) * m + i) * 3;
    vedt_sphere_result r;
    int v[3];
    const bool inside = voxel_coord(c[0], M.o[0], M.vs, M.X, v[0]) && voxel_coord(c[1], M.o[1], M.vs, M.Y, v[1]) &&
                        voxel_coord(c[2], M.o[2], M.vs, M.Z, v[2]);
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
    const int64_t id = v[0] + static_cast<int64_t>(M.X) * (v[1] + static_cast<int64_t>(M.Y) * v[2]);
    r.sqdist = M.sq[g][id];
    r.idx = M.ix[g][id];
    if (r.idx < 0) {
        r.dist = __int_as_float(0x7f800000);
        r.clearance = r.dist;
        r.nearest[0] = r.nearest[1] = r.nearest[2] = __int_as_float(0x7fc00000);
        r.status = VEDT_SPHERE_EMPTY;
        out[t] = r;
        return;
    }
    r.dist = __fmul_rn(M.vs, __fsqrt_rn(static_cast<float>(r.sqdist)));
    r.clearance = __fsub_rn(r.dist, radii[i]);
    const int j = r.idx;
    const int nv[3] = {j % M.X, (j / M.X) % M.Y, j / (M.X * M.Y)};
    for (int a = 0; a < 3; ++a)
        r.nearest[a] = __fadd_rn(M.o[a], __fmul_rn(__fadd_rn(static_cast<float>(nv[a]), 0.5f), M.vs));
    r.status = VEDT_SPHERE_OK;
    out[t] = r;
}

vedt_status from_cuda(cudaError_t e) {
    return e == cudaSuccess ? VEDT_OK : (e == cudaErrorMemoryAllocation ? VEDT_ENOMEM : VEDT_ECUDA);
}

#define BCHECK(call)                                 \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

}  // namespace

namespace vedt {
vedt_status build_table(GridTable &t, const std::vector<GridDesc> &grids, void *dev_desc, void *dev_tmaps,
                        int32_t *err, int pzx);
}

struct vedt_batch {
    std::vector<vedt_map *> maps;
    cudaStream_t stream = nullptr;
    // EDT tables: [0] grids of maps with every dim <= 256, [1] the others
    GridTable tab[2];
    int ngrid[2] = {0, 0};
    void *tab_mem = nullptr;
    unsigned *counters = nullptr;       // per table: next, done_x[n], done_y[n]
    size_t counter_bytes = 0;
    int32_t *err = nullptr;
    int ctas_per_sm = 0, rows_per_item = 32, persistent = 1;
    int bands = 0;                       // bands per line of passes Y and Z (0: default)
    int pzx = 0;                         // pass-Z tile width of the small table (0: default)
    int which = VEDT_MAP_BOTH;           // grids the EDT covers
    // pipeline
    MapRef *refs = nullptr;
    float *link_pts = nullptr;
    uint8_t *link_of = nullptr;
    int64_t n_link_pts = 0;
    int n_links = 0;
    float *poses = nullptr;             // [n][VEDT_MAX_LINKS][12]
    int64_t *offs = nullptr;            // [n + 1]
    const float *xyz = nullptr;
    int64_t max_points_per_map = 0;
    uint32_t link_mask = 0;
    const float *centres = nullptr, *radii = nullptr;
    int m = 0;
    vedt_sphere_result *out = nullptr;
    bool frame_set = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void free_batch(vedt_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->tab_mem);
    cudaFree(b->counters);
    cudaFree(b->err);
    cudaFree(b->refs);
    cudaFree(b->link_pts);
    cudaFree(b->link_of);
    cudaFree(b->poses);
    cudaFree(b->offs);
    delete b;
}

GridDesc grid_desc(const vedt_map *m, int i) {
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
    return g;
}

// (re)builds the per-mode tables, including the persistent pass-X item prefixes
vedt_status build_tables(vedt_batch *b) {
    std::vector<GridDesc> mode[2];
    for (vedt_map *m : b->maps)
        for (int i = 0; i < 2; ++i)
            if (b->which & (1 << i)) mode[m->large].push_back(grid_desc(m, i));
    char *base = static_cast<char *>(b->tab_mem);
    size_t off = 0;
    for (int md = 0; md < 2; ++md) {
        b->ngrid[md] = static_cast<int>(mode[md].size());
        if (mode[md].empty()) continue;
        int64_t xi = 0;
        for (GridDesc &g : mode[md]) {
            g.xi_begin = xi;
            xi += (static_cast<int64_t>(g.Y) * g.Z + b->rows_per_item - 1) / b->rows_per_item;
        }
        const size_t nd = mode[md].size();
        char *desc = base + off;
        off += (sizeof(GridDesc) * nd + 127) / 128 * 128;
        char *tm = base + off;
        off += sizeof(CUtensorMap) * 2 * nd;
        // the large-grid table keeps 32 x 1 pass-Z tiles, the shape of its persistent kernel
        vedt_status st = build_table(b->tab[md], mode[md], desc, tm, b->err, md == 0 ? b->pzx : kEnvCols);
        if (st != VEDT_OK) return st;
        b->tab[md].bands = md == 0 ? b->bands : ((b->bands == 4 || b->bands == 8) ? b->bands : 0);
    }
    return VEDT_OK;
}

}  // namespace

extern "C" {

vedt_status vedt_batch_create(vedt_map *const *maps, int n, void *stream, vedt_batch **out) {
    if (!maps || !out || n < 1) return VEDT_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!maps[i]) return VEDT_EINVAL;
    vedt_batch *b = new (std::nothrow) vedt_batch();
    if (!b) return VEDT_ENOMEM;
    b->maps.assign(maps, maps + n);
    b->stream = static_cast<cudaStream_t>(stream);
    const size_t ng = 2 * static_cast<size_t>(n);
    cudaError_t e = cudaMalloc(&b->tab_mem, (sizeof(GridDesc) + 2 * sizeof(CUtensorMap)) * ng + 1024);
    b->counter_bytes = sizeof(unsigned) * (2 + 2 * ng);
    if (e == cudaSuccess) e = cudaMalloc(&b->counters, b->counter_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->refs, sizeof(MapRef) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->poses, sizeof(float) * n * VEDT_MAX_LINKS * 12);
    if (e == cudaSuccess) e = cudaMalloc(&b->offs, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMemset(b->poses, 0, sizeof(float) * n * VEDT_MAX_LINKS * 12);
    if (e != cudaSuccess) {
        free_batch(b);
        return from_cuda(e);
    }
    std::vector<MapRef> refs(n);
    for (int i = 0; i < n; ++i) {
        const vedt_map *m = maps[i];
        MapRef &r = refs[i];
        for (int g = 0; g < 2; ++g) {
            r.occ[g] = m->occ[g];
            r.sq[g] = m->sq[g];
            r.ix[g] = m->ix[g];
        }
        r.X = m->X;
        r.Y = m->Y;
        r.Z = m->Z;
        r.vs = m->vs;
        for (int a = 0; a < 3; ++a) r.o[a] = m->origin[a];
        r.N = m->N;
    }
    e = cudaMemcpy(b->refs, refs.data(), sizeof(MapRef) * n, cudaMemcpyHostToDevice);
    vedt_status st = from_cuda(e);
    if (st == VEDT_OK) st = build_tables(b);
    if (st != VEDT_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return VEDT_OK;
}

vedt_status vedt_batch_destroy(vedt_batch *b) {
    if (!b) return VEDT_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return VEDT_OK;
}

vedt_status vedt_batch_set_tuning(vedt_batch *b, int ctas_per_sm, int rows_per_item, int persistent) {
    if (!b || ctas_per_sm < 0 || rows_per_item < 1 || rows_per_item > 4096) return VEDT_EINVAL;
    BCHECK(cudaStreamSynchronize(b->stream));
    b->ctas_per_sm = ctas_per_sm;
    b->persistent = persistent ? 1 : 0;
    if (rows_per_item != b->rows_per_item) {
        b->rows_per_item = rows_per_item;
        vedt_status st = build_tables(b);
        if (st != VEDT_OK) return st;
    }
    if (b->exec) {   // a recorded graph holds the old launch shapes
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return VEDT_OK;
}

vedt_status vedt_batch_set_bands(vedt_batch *b, int bands) {
    if (!b || !(bands == 0 || bands == 1 || bands == 2 || bands == 4 || bands == 8)) return VEDT_EINVAL;
    BCHECK(cudaStreamSynchronize(b->stream));
    b->bands = bands;
    b->tab[0].bands = bands;
    b->tab[1].bands = (bands == 4 || bands == 8) ? bands : 0;
    if (b->exec) {   // a recorded graph holds the old launches
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return VEDT_OK;
}

vedt_status vedt_batch_set_tile_z(vedt_batch *b, int cols_x) {
    if (!b || !(cols_x == 0 || cols_x == 8 || cols_x == 32)) return VEDT_EINVAL;
    BCHECK(cudaStreamSynchronize(b->stream));
    b->pzx = cols_x;
    if (b->exec) {   // a recorded graph holds the old launch shapes
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return build_tables(b);
}

int vedt_batch_tile_z(const vedt_batch *b) { return b && b->ngrid[0] ? b->tab[0].pzx : 0; }

vedt_status vedt_batch_set_grids(vedt_batch *b, int which) {
    if (!b || (which != VEDT_MAP_ENV && which != VEDT_MAP_SELF && which != VEDT_MAP_BOTH)) return VEDT_EINVAL;
    BCHECK(cudaStreamSynchronize(b->stream));
    b->which = which;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return build_tables(b);
}

// A batch writes its maps' fields without their incremental snapshots: the next EDT of
// an incremental map recomputes.
static void invalidate_snapshots(vedt_batch *b) {
    for (vedt_map *m : b->maps) m->snap_valid[0] = m->snap_valid[1] = false;
}

vedt_status vedt_batch_compute_edt(vedt_batch *b) {
    if (!b) return VEDT_EINVAL;
    invalidate_snapshots(b);
    for (int md = 0; md < 2; ++md) {
        if (b->ngrid[md] == 0) continue;
        const GridTable &t = b->tab[md];
        if (b->persistent) {
            unsigned *base = b->counters + (md == 0 ? 0 : 1 + 2 * b->ngrid[0]);
            BCHECK(cudaMemsetAsync(base, 0, sizeof(unsigned) * (1 + 2 * b->ngrid[md]), b->stream));
            PersistCounters c{};
            c.next = base;
            c.done_x = base + 1;
            c.done_y = base + 1 + b->ngrid[md];
            int64_t nx = 0;
            const int gpm = (b->which == VEDT_MAP_BOTH) ? 2 : 1;
            for (vedt_map *m : b->maps)
                if (m->large == md)
                    nx += gpm * ((static_cast<int64_t>(m->Y) * m->Z + b->rows_per_item - 1) / b->rows_per_item);
            c.n_x = static_cast<unsigned>(nx);
            c.n_y = static_cast<unsigned>(t.tiles_y);
            c.n_z = static_cast<unsigned>(t.tiles_z);
            BCHECK(launch_persistent(t, c, b->ctas_per_sm, b->rows_per_item, b->stream));
        } else {
            BCHECK(launch_pass_x(t, b->stream));
            BCHECK(launch_pass_y(t, b->stream));
            BCHECK(launch_pass_z(t, b->stream));
        }
    }
    return VEDT_OK;
}

vedt_status vedt_batch_register_links(vedt_batch *b, int n_links, const float *const *xyz, const int64_t *n_vox) {
    if (!b || n_links < 1 || n_links > VEDT_MAX_LINKS || !xyz || !n_vox) return VEDT_EINVAL;
    int64_t total = 0;
    for (int k = 0; k < n_links; ++k) {
        if (n_vox[k] < 0 || (n_vox[k] > 0 && !xyz[k])) return VEDT_EINVAL;
        total += n_vox[k];
    }
    std::vector<float> pts(static_cast<size_t>(total) * 3);
    std::vector<uint8_t> of(static_cast<size_t>(total));
    int64_t w = 0;
    for (int k = 0; k < n_links; ++k) {
        for (int64_t i = 0; i < n_vox[k]; ++i) {
            for (int a = 0; a < 3; ++a) pts[3 * (w + i) + a] = xyz[k][3 * i + a];
            of[w + i] = static_cast<uint8_t>(k);
        }
        w += n_vox[k];
    }
    BCHECK(cudaStreamSynchronize(b->stream));
    cudaFree(b->link_pts);
    cudaFree(b->link_of);
    b->link_pts = nullptr;
    b->link_of = nullptr;
    b->n_link_pts = 0;
    if (total > 0) {
        BCHECK(cudaMalloc(&b->link_pts, pts.size() * sizeof(float)));
        BCHECK(cudaMalloc(&b->link_of, of.size()));
        BCHECK(cudaMemcpy(b->link_pts, pts.data(), pts.size() * sizeof(float), cudaMemcpyHostToDevice));
        BCHECK(cudaMemcpy(b->link_of, of.data(), of.size(), cudaMemcpyHostToDevice));
    }
    b->n_link_pts = total;
    b->n_links = n_links;
    return VEDT_OK;
}

vedt_status vedt_batch_set_frame(vedt_batch *b, const float *xyz_dev, const int64_t *offsets_host,
                                 const float *poses_host, uint32_t link_mask, const float *centres_dev,
                                 const float *radii_dev, int m, vedt_sphere_result *out_dev) {
    const int n = b ? static_cast<int>(b->maps.size()) : 0;
    if (!b || !offsets_host || !poses_host || m < 0 || m > kMaxQuery) return VEDT_EINVAL;
    if (m > 0 && (!centres_dev || !radii_dev || !out_dev)) return VEDT_EINVAL;
    if (offsets_host[0] != 0) return VEDT_EINVAL;
    int64_t mx = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t c = offsets_host[i + 1] - offsets_host[i];
        if (c < 0) return VEDT_EINVAL;
        mx = std::max(mx, c);
    }
    if (offsets_host[n] > 0 && !xyz_dev) return VEDT_EINVAL;
    if (b->n_links < 32 && (link_mask >> b->n_links) != 0u) return VEDT_EINVAL;
    if (b->exec && (xyz_dev != b->xyz || centres_dev != b->centres || radii_dev != b->radii || out_dev != b->out ||
                    m != b->m || mx > b->max_points_per_map || link_mask != b->link_mask))
        return VEDT_EINVAL;   // a recorded graph holds these buffers and launch shapes
    std::vector<float> P(static_cast<size_t>(n) * VEDT_MAX_LINKS * 12, 0.f);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < b->n_links; ++k)
            std::memcpy(&P[(static_cast<size_t>(i) * VEDT_MAX_LINKS + k) * 12],
                        poses_host + (static_cast<size_t>(i) * b->n_links + k) * 12, sizeof(float) * 12);
    BCHECK(cudaMemcpyAsync(b->poses, P.data(), sizeof(float) * P.size(), cudaMemcpyHostToDevice, b->stream));
    BCHECK(cudaMemcpyAsync(b->offs, offsets_host, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, b->stream));
    BCHECK(cudaStreamSynchronize(b->stream));   // host staging above is freed on return
    b->xyz = xyz_dev;
    if (!b->exec) b->max_points_per_map = mx;
    b->link_mask = link_mask;
    b->centres = centres_dev;
    b->radii = radii_dev;
    b->m = m;
    b->out = out_dev;
    b->frame_set = true;
    return VEDT_OK;
}

vedt_status vedt_batch_run(vedt_batch *b) {
    if (!b || !b->frame_set) return VEDT_EINVAL;
    const int n = static_cast<int>(b->maps.size());
    int64_t nmax = 0;
    for (vedt_map *m : b->maps) nmax = std::max(nmax, m->N);
    const int sms = sm_count();
    {
        const int64_t want = (nmax / 16 + 255) / 256;
        const int bx = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, std::max(1, 2 * sms / n + 1))));
        k_clear_many<<<dim3(bx, 2 * n), 256, 0, b->stream>>>(b->refs);
        BCHECK(cudaGetLastError());
    }
    if (b->n_link_pts > 0 && b->link_mask) {
        const int bx = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((b->n_link_pts + 255) / 256, 64)));
        k_insert_links_many<<<dim3(bx, n), 256, 0, b->stream>>>(b->refs, b->link_pts, b->link_of, b->n_link_pts,
                                                                  b->poses, b->link_mask);
        BCHECK(cudaGetLastError());
    }
    if (b->max_points_per_map > 0) {
        const int bx = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((b->max_points_per_map + 255) / 256, 64)));
        k_insert_points_many<<<dim3(bx, n), 256, 0, b->stream>>>(b->refs, b->xyz, b->offs);
        BCHECK(cudaGetLastError());
    }
    vedt_status st = vedt_batch_compute_edt(b);
    if (st != VEDT_OK) return st;
    if (b->m > 0) {
        const int64_t tot = static_cast<int64_t>(n) * 2 * b->m;
        k_query_many<<<static_cast<unsigned>((tot + 127) / 128), 128, 0, b->stream>>>(b->refs, n, b->centres, b->radii,
                                                                                      b->m, b->out);
        BCHECK(cudaGetLastError());
    }
    return VEDT_OK;
}

vedt_status vedt_batch_capture(vedt_batch *b) {
    if (!b || !b->frame_set || !b->stream) return VEDT_EINVAL;   // capture needs a non-default stream
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    BCHECK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    vedt_status st = vedt_batch_run(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != VEDT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    BCHECK(e);
    b->graph = g;
    BCHECK(cudaGraphInstantiate(&b->exec, g, 0));
    return VEDT_OK;
}

vedt_status vedt_batch_replay(vedt_batch *b) {
    if (!b || !b->exec) return VEDT_EINVAL;
    invalidate_snapshots(b);
    BCHECK(cudaGraphLaunch(b->exec, b->stream));
    return VEDT_OK;
}

vedt_status vedt_batch_check(vedt_batch *b) {
    if (!b) return VEDT_EINVAL;
    BCHECK(cudaStreamSynchronize(b->stream));
    int32_t e = 0;
    BCHECK(cudaMemcpy(&e, b->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) {
        BCHECK(cudaMemset(b->err, 0, sizeof(int32_t)));
        return (e & kErrTimeout) ? VEDT_ETIMEOUT : VEDT_ECUDA;
    }
    return VEDT_OK;
}

}  // extern "C"
