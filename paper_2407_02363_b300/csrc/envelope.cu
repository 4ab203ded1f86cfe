// Stand-alone kernels of passes Y and Z (one tile per CTA; the tile code and its design are
// in envelope.cuh).  Grids with every dimension <= 256 take the small word sizes (PolY /
// PolZ, 1, 2, 4 or 8 bands), tables with a larger grid the large ones (PolYL / PolZL, four
// or eight bands).
#include "envelope.cuh"

namespace vedt {
namespace lenv {

template <int NB, class P>
__global__ void __launch_bounds__(NB * 32) k_env_y(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                                   int ng, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_tile_grid(gd, ng, t, false);
    const GridDesc &G = gd[g];
    const Layout<NB, P> L(G.Y);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // row sites and row flags come from pass X
    if (G.changed && *G.changed == 0) return;   // unchanged since its last EDT
    tile_y<NB, true, P>(G, &tm[2 * g], static_cast<int>(t - G.ty_begin), smem, bar, 0, err);
}

template <int NB, int PX, class P>
__global__ void __launch_bounds__(NB * 32) k_env_z(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                                   int ng, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_tile_grid(gd, ng, t, true);
    const GridDesc &G = gd[g];
    const Layout<NB, P> L(G.Z);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // the 2-D sites and slice flags come from pass Y
    if (G.changed && *G.changed == 0) return;   // unchanged since its last EDT
    tile_z<NB, true, PX, P>(G, &tm[2 * g + 1], static_cast<int>(t - G.tz_begin), smem, bar, 0, err);
}

template <int NB, class P>
static cudaError_t launch_y(const GridTable &t, cudaStream_t s) {
    const size_t sm = static_cast<size_t>(Layout<NB, P>(t.maxY).bytes);
    const cudaError_t e = ensure_dyn_smem<k_env_y<NB, P>>(sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_env_y<NB, P>, dim3(static_cast<unsigned>(t.tiles_y)), dim3(NB * 32), sm, s, t.desc, t.tmaps,
                      t.n, t.err);
}

template <int NB, int PX, class P>
static cudaError_t launch_z(const GridTable &t, cudaStream_t s) {
    const size_t sm = static_cast<size_t>(Layout<NB, P>(t.maxZ).bytes);
    const cudaError_t e = ensure_dyn_smem<k_env_z<NB, PX, P>>(sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_env_z<NB, PX, P>, dim3(static_cast<unsigned>(t.tiles_z)), dim3(NB * 32), sm, s, t.desc,
                      t.tmaps, t.n, t.err);
}

template <int PX>
static cudaError_t launch_z_bands(const GridTable &t, int bands, cudaStream_t s) {
    if (t.large) return bands == 8 ? launch_z<8, PX, PolZL>(t, s) : launch_z<4, PX, PolZL>(t, s);
    switch (bands) {
        case 1: return launch_z<1, PX, PolZ>(t, s);
        case 2: return launch_z<2, PX, PolZ>(t, s);
        case 8: return launch_z<8, PX, PolZ>(t, s);
        default: return launch_z<4, PX, PolZ>(t, s);
    }
}

}  // namespace lenv

cudaError_t launch_env_y(const GridTable &t, int bands, cudaStream_t s) {
    if (t.tiles_y == 0) return cudaSuccess;
    if (t.large) return bands == 8 ? lenv::launch_y<8, lenv::PolYL>(t, s) : lenv::launch_y<4, lenv::PolYL>(t, s);
    switch (bands) {
        case 1: return lenv::launch_y<1, lenv::PolY>(t, s);
        case 2: return lenv::launch_y<2, lenv::PolY>(t, s);
        case 8: return lenv::launch_y<8, lenv::PolY>(t, s);
        default: return lenv::launch_y<4, lenv::PolY>(t, s);
    }
}

cudaError_t launch_env_z(const GridTable &t, int bands, cudaStream_t s) {
    if (t.tiles_z == 0) return cudaSuccess;
    if (t.pzx == 8) return lenv::launch_z_bands<8>(t, bands, s);
    if (t.pzx == 32) return lenv::launch_z_bands<32>(t, bands, s);
    return cudaErrorInvalidValue;   // the table's tiles were counted for another shape
}

}  // namespace vedt
