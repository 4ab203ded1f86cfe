// Internal declarations shared by the CUDA translation units of libvedt.
#pragma once
#include <atomic>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vedt.h"

namespace vedt {

constexpr int kTile = 32;            // lanes per warp
constexpr int kEnvCols = 32;         // columns per pass-Y/Z tile (one warp per band of the lines)
constexpr int kBox = 256;            // max TMA box extent along one dimension
constexpr uint16_t kNoX = 0xFFFF;    // pass-X "row has no site"
constexpr int kSmallMax = 256;       // all dims <= 256: 16-bit packed 2-D sites, 8-bit links
// Pass-Z tile: a patch of px x (32 / px) columns (x fastest), one lane per column, px = 8
// or 32 (GridTable::pzx; a batch's table of grids above 256 keeps 32, the shape of its
// persistent kernel).  Columns close in both x and y have similar
// envelopes along z, so an 8 x 4 patch keeps the lanes of a warp in step more often than a
// 32 x 1 row; a row writes whole 128-byte lines of the field where an 8-wide run of a grid
// whose X is no multiple of 8 straddles two 32-byte sectors.
inline int64_t small_tiles_z(int Xp, int Y, int px) {
    const int py = kEnvCols / px;
    return static_cast<int64_t>(Xp / px) * ((Y + py - 1) / py);
}

// error word bits (device-side guards)
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;

// One grid in an EDT launch.  Intermediates use a padded pitch Xp (multiple of 32) so
// every tile is whole and every TMA row stride is a multiple of 16 bytes.
struct GridDesc {
    const uint8_t *occ;     // [Z][Y][X] occupancy
    void *xs;               // [Z][Y][Xp] pass-X nearest site x: small uint8 (valid iff
                            // row_has), large uint16 (kNoX if the row is empty)
    uint8_t *row_has;       // [Z][Y] small mode: 1 iff row (y, z) has an occupied voxel
    void *s2;               // [Z][Y][Xp] pass-Y 2-D site: small x | y << 8, large x | y << 16
    uint8_t *slice_has;     // [Z] 1 iff slice z has an occupied voxel
    int32_t *sqdist;        // [Z][Y][X]
    int32_t *idx;           // [Z][Y][X]
    int32_t X, Y, Z, Xp;
    int64_t row_begin;      // prefix over rows (Y*Z) of the grids before this one
    int64_t ty_begin;       // prefix over pass-Y tiles ((Xp/32)*Z)
    int64_t tz_begin;       // prefix over pass-Z tiles (small_tiles_z)
    int64_t xi_begin;       // prefix over persistent pass-X items (ceil(Y*Z / rows_per_item))
    const uint32_t *changed;  // NULL, or a device word: 0 = occupancy unchanged since this
                              // grid's last EDT (incremental maps), so the passes skip it
};

// Work counters of one persistent EDT launch (device memory, zeroed before the launch).
struct PersistCounters {
    unsigned *next;         // next work item
    unsigned *done_x;       // [n grids] pass-X items finished
    unsigned *done_y;       // [n grids] pass-Y tiles finished
    unsigned n_x, n_y, n_z; // item counts per pass
};

struct GridTable {
    GridDesc *desc;              // device array [n]
    CUtensorMap *tmaps;          // device array [2n]: {xs box (32, by, 1), s2 box (pzx, 32 / pzx, bz)}
    int n;
    int large;                   // 0: every grid has dims <= 256
    int maxY, maxZ, maxXp;
    int64_t rows, tiles_y, tiles_z;
    int32_t *err;                // device error word
    int bands;                   // bands per line in passes Y and Z (0: the default)
    int pzx;                     // pass-Z tile width in x, 8 or 32 (see small_tiles_z)
    int incr;                    // 1: pass X honours GridDesc::changed (incremental maps)
};

// Launch with programmatic stream serialization: the kernel may start while the previous
// kernel on the stream finishes, and orders itself with pdl_wait() (griddepcontrol.wait)
// before touching anything that kernel reads or writes.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes`, calling the runtime
// only when the limit grows (the attribute call costs far more host time than a launch).
template <auto Kernel>
cudaError_t ensure_dyn_smem(size_t bytes) {
    static std::atomic<size_t> have{0};
    if (bytes <= have.load(std::memory_order_acquire)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
    size_t h = have.load(std::memory_order_acquire);
    while (h < bytes && !have.compare_exchange_weak(h, bytes, std::memory_order_acq_rel)) {
    }
    return cudaSuccess;
}

// host-side helpers (api.cu)
CUresult encode_tmap(CUtensorMap *m, CUtensorMapDataType t, int elem, void *base,
                     uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1, uint32_t b2);
// Pass-Z tile width of a table when none is set: 8 x 4 patches if every grid's X is a
// multiple of 8 (whole 32-byte sectors per run), else 32 x 1 rows.
int default_pzx(const GridDesc *grids, size_t n);

// SM count of the current device, cached per device (insert.cu)
int sm_count();

// launchers (edt.cu)
// logodds (non-null: small-mode tables of one grid only) = that grid's log-odds, updated
// by pass X from the occupancy before the rows are swept; lo_param = {l_hit, l_miss,
// l_min, l_max, threshold}
cudaError_t launch_pass_x(const GridTable &t, cudaStream_t s, int8_t *logodds = nullptr,
                          const int *lo_param = nullptr);
cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s);
cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s);
// small-mode envelope passes (envelope.cu), `bands` per line = 1, 2, 4 or 8
cudaError_t launch_env_y(const GridTable &t, int bands, cudaStream_t s);
cudaError_t launch_env_z(const GridTable &t, int bands, cudaStream_t s);   // tile shape t.pzx
cudaError_t launch_persistent(const GridTable &t, const PersistCounters &c, int ctas_per_sm, int rows_per_item,
                              cudaStream_t s);
cudaError_t launch_wait_selftest(const unsigned *counter, uint32_t limit, int32_t *err, cudaStream_t s);

// launchers (insert.cu)
struct LinkPose { float T[VEDT_MAX_LINKS][12]; };
cudaError_t launch_clear(uint8_t *p, int64_t n, cudaStream_t s);
cudaError_t launch_logodds(uint8_t *occ, int8_t *L, int64_t n, const int (&p)[5], cudaStream_t s);
cudaError_t launch_occ_diff(const uint8_t *occ, uint8_t *snap, uint32_t *changed, int64_t n_al, int grids,
                            cudaStream_t s);
cudaError_t launch_insert_points(uint8_t *env, const uint8_t *self, int X, int Y, int Z, float vs,
                                 const float *origin, const float *xyz, int64_t n, const float *T,
                                 int filter_self, const uint8_t *keep, int64_t *counts, cudaStream_t s);
cudaError_t launch_insert_links(uint8_t *self, int X, int Y, int Z, float vs, const float *origin,
                                const float *pts, const uint8_t *link_of, int64_t n,
                                const LinkPose &poses, uint32_t mask, cudaStream_t s);
struct QueryGrid { const int32_t *sqdist; const int32_t *idx; };
cudaError_t launch_query(const QueryGrid *g, int ng, int X, int Y, int Z, float vs,
                         const float *origin, const float *centres, const float *radii, int m,
                         vedt_sphere_result *out, cudaStream_t s);

}  // namespace vedt

#include <vector>

namespace vedt {
constexpr int kMaxQuery = 4096;
constexpr int kQRing = 4;   // host frames' page-locked query-input slots
struct EvPair {
    int kind;
    cudaEvent_t a, b;
};
}  // namespace vedt

// A map handle: the environment grid M_I ([0]) and self grid M_S ([1]), their fields
// and EDT scratch, all owned.
struct vedt_map {
    using GridTable = vedt::GridTable;
    using QueryGrid = vedt::QueryGrid;
    using EvPair = vedt::EvPair;
    int32_t X = 0, Y = 0, Z = 0, Xp = 0;
    float vs = 0.f;
    float origin[3] = {0, 0, 0};
    cudaStream_t stream = nullptr;
    int large = 0;
    int64_t N = 0;
    // [0] = environment M_I, [1] = self M_S
    uint8_t *occ[2] = {nullptr, nullptr};
    int32_t *sq[2] = {nullptr, nullptr};
    int32_t *ix[2] = {nullptr, nullptr};
    void *xs[2] = {nullptr, nullptr};
    uint8_t *row_has[2] = {nullptr, nullptr};
    void *s2[2] = {nullptr, nullptr};
    uint8_t *slice_has[2] = {nullptr, nullptr};
    int32_t *err = nullptr;
    // incremental EDT: per grid, 1 iff the last vedt_compute_edt recomputed it (always 1
    // unless incremental); snapshot of each grid's occupancy at its last EDT (both grids
    // in one allocation, same layout as occ)
    uint32_t *changed = nullptr;
    uint8_t *snap = nullptr;
    // Bayesian occupancy of M_I: int8 log-odds per voxel (layout of the occupancy) and
    // the update's parameters {l_hit, l_miss, l_min, l_max, threshold}
    int8_t *logodds = nullptr;
    int lo_param[5] = {0, 0, 0, 0, 0};
    bool fuse_lo = false;   // set by vedt_frame: the M_I EDT's pass X applies the update
    int incremental = 0;
    bool snap_valid[2] = {false, false};   // fields match the snapshot (host view)
    // EDT launch tables for which = ENV (0), SELF (1), BOTH (2)
    GridTable tab[3];
    void *tab_mem = nullptr;
    // query scratch
    QueryGrid *qgrids = nullptr;   // device [3]: env, self, env+self ... see below
    float *q_in = nullptr;         // device centres (3*kMaxQuery) + radii (kMaxQuery) of vedt_query_spheres
    vedt_sphere_result *q_out = nullptr;
    // links
    float *link_pts = nullptr;
    uint8_t *link_of = nullptr;
    // host frames: two device staging buffers for point clouds, filled on a copy stream
    // so that the next frame's upload overlaps this frame's kernels
    float *stage[2] = {nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;
    // frames: the self map's EDT runs on a side stream, concurrently with the point
    // insertion and the environment map's EDT
    cudaStream_t side_stream = nullptr;
    cudaEvent_t links_done = nullptr, self_done = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};    // upload into stage[b] finished
    // The sphere centres and radii of host frame h are copied on the host into page-locked
    // slot h % kQRing (the layout of a q_in area), which that frame's query kernel reads
    // in place: 16 bytes per sphere over the bus instead of two small uploads, which cost
    // a frame about 36 us of latency even on a stream of their own.
    float *pin_q = nullptr;                       // kQRing slots
    const float *pin_q_dev = nullptr;             // the same memory as the device addresses it
    cudaEvent_t fdone[vedt::kQRing] = {};         // host frame h finished (slot h % kQRing)
    int64_t hframes = 0;                          // host frames queued
    cudaEvent_t done = nullptr;    // completion of the last asynchronous host frame
    int64_t stage_cap = 0;         // points per staging buffer
    int64_t n_link_pts = 0;
    int n_links = 0;
    // timing
    bool timing = false;
    std::vector<EvPair> pending;
    std::vector<cudaEvent_t> free_events;
    double ms[VEDT_NUM_KERNELS] = {};
    int64_t cnt[VEDT_NUM_KERNELS] = {};
};


// ---------------------------------------------------------------------------------
// device helpers: mbarrier + TMA (sm_90+ PTX, used here on sm_103a)
// ---------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace vedt {

// World point -> voxel along one axis: floor((p - o) / vs) in fp32 with explicitly
// rounded subtraction and division; inside iff 0 <= v < n (NaN is outside).
__device__ __forceinline__ bool voxel_coord(float p, float o, float vs, int n, int &v) {
    const float f = floorf(__fdiv_rn(__fsub_rn(p, o), vs));
    if (!(f >= 0.0f) || !(f < static_cast<float>(n))) return false;
    v = static_cast<int>(f);
    return true;
}

// w_a = ((T_a0 p_x + T_a1 p_y) + T_a2 p_z) + T_a3 in fp32, every step rounded, no FMA.
__device__ __forceinline__ void rigid(const float *T, float px, float py, float pz, float &wx, float &wy, float &wz) {
    wx = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T[0], px), __fmul_rn(T[1], py)), __fmul_rn(T[2], pz)), T[3]);
    wy = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T[4], px), __fmul_rn(T[5], py)), __fmul_rn(T[6], pz)), T[7]);
    wz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(T[8], px), __fmul_rn(T[9], py)), __fmul_rn(T[10], pz)), T[11]);
}

// Programmatic dependent launch: let the next kernel on the stream start launching (every
// block calls it first thing; the dependent still waits for this grid to finish), and wait
// for the previous kernel's grid to complete with its memory visible.  Both are no-ops in
// a launch without programmatic serialization.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Ends the barrier's life so that its bytes can hold other data (after every wait on it).
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Debug builds (-DVEDT_DEBUG_BOUNDS, libvedt_debug.so) check the indices the EDT passes
// compute against their buffers: a bad one sets kErrBounds in the error word (reported by
// vedt_check as VEDT_ECUDA) and its access is skipped.  Release builds drop the checks.
#ifdef VEDT_DEBUG_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif

__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int32_t *err) {
    if constexpr (!kCheckBounds) return true;
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, kErrBounds);
    return false;
}

// Log-odds occupancy of M_I (Sec. III-A, integer log-odds reading): a hit adds l_hit, a
// miss subtracts l_miss, the sum is clamped to [l_min, l_max]; occupied iff >= threshold.
struct LogOdds { int hit, miss, lo, hi, thr; };

__device__ __forceinline__ int logodds_step(int L, bool hit, const LogOdds &p) {
    return min(max(L + (hit ? p.hit : -p.miss), p.lo), p.hi);
}

// Bounded wait: gives up after `limit` polls (each try_wait already suspends for a
// hardware-chosen interval), flags kErrTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err,
                                                  uint32_t limit = 1u << 22) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, kErrTimeout);
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace vedt
#endif
