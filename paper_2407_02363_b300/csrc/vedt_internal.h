// Internal declarations shared by the CUDA translation units of libvedt.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vedt.h"

namespace vedt {

constexpr int kTile = 32;            // lanes per warp
constexpr int kEnvCols = 32;         // columns per pass-Y/Z tile (two warps: lower / upper half)
constexpr int kBox = 256;            // max TMA box extent along one dimension
constexpr uint16_t kNoX = 0xFFFF;    // pass-X "row has no site"
constexpr int kSmallMax = 256;       // all dims <= 256: 16-bit packed 2-D sites, 8-bit links

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
    int64_t tz_begin;       // prefix over pass-Z tiles ((Xp/32)*Y)
};

struct GridTable {
    GridDesc *desc;              // device array [n]
    CUtensorMap *tmaps;          // device array [2n]: {xs box (32, by, 1), s2 box (32, 1, bz)}
    int n;
    int large;                   // 0: every grid has dims <= 256
    int maxY, maxZ, maxXp;
    int64_t rows, tiles_y, tiles_z;
    int32_t *err;                // device error word
};

// host-side helpers (api.cu)
CUresult encode_tmap(CUtensorMap *m, CUtensorMapDataType t, int elem, void *base,
                     uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1, uint32_t b2);

// launchers (edt.cu)
cudaError_t launch_pass_x(const GridTable &t, cudaStream_t s);
cudaError_t launch_pass_y(const GridTable &t, cudaStream_t s);
cudaError_t launch_pass_z(const GridTable &t, cudaStream_t s);

// launchers (insert.cu)
struct LinkPose { float T[VEDT_MAX_LINKS][12]; };
cudaError_t launch_clear(uint8_t *p, int64_t n, cudaStream_t s);
cudaError_t launch_insert_points(uint8_t *env, const uint8_t *self, int X, int Y, int Z, float vs,
                                 const float *origin, const float *xyz, int64_t n, const float *T,
                                 int filter_self, int64_t *counts, cudaStream_t s);
cudaError_t launch_insert_links(uint8_t *self, int X, int Y, int Z, float vs, const float *origin,
                                const float *pts, const uint8_t *link_of, int64_t n,
                                const LinkPose &poses, uint32_t mask, cudaStream_t s);
struct QueryGrid { const int32_t *sqdist; const int32_t *idx; };
cudaError_t launch_query(const QueryGrid *g, int ng, int X, int Y, int Z, float vs,
                         const float *origin, const float *centres, const float *radii, int m,
                         vedt_sphere_result *out, cudaStream_t s);

}  // namespace vedt

// ---------------------------------------------------------------------------------
// device helpers: mbarrier + TMA (sm_90+ PTX, used here on sm_103a)
// ---------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace vedt {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
