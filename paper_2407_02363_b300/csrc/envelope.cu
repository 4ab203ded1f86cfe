// Stand-alone kernels of passes Y and Z for grids whose every dimension is at most 256
// (one tile per CTA; the tile code and its design are in envelope.cuh).
#include "envelope.cuh"

namespace vedt {
namespace lenv {

template <int NB>
__global__ void __launch_bounds__(NB * 32) k_env_y(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                                   int ng, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_tile_grid(gd, ng, t, false);
    const GridDesc &G = gd[g];
    const Layout<NB, uint8_t> L(G.Y);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // row sites and row flags come from pass X
    if (G.changed && *G.changed == 0) return;   // unchanged since its last EDT
    tile_y<NB, true>(G, &tm[2 * g], static_cast<int>(t - G.ty_begin), smem, bar, 0, err);
}

template <int NB, int PX>
__global__ void __launch_bounds__(NB * 32) k_env_z(const GridDesc *__restrict__ gd, const CUtensorMap *__restrict__ tm,
                                                   int ng, int32_t *err) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_trigger();
    const int64_t t = blockIdx.x;
    const int g = find_tile_grid(gd, ng, t, true);
    const GridDesc &G = gd[g];
    const Layout<NB, uint16_t> L(G.Z);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();   // the 2-D sites and slice flags come from pass Y
    if (G.changed && *G.changed == 0) return;   // unchanged since its last EDT
    tile_z<NB, true, PX>(G, &tm[2 * g + 1], static_cast<int>(t - G.tz_begin), smem, bar, 0, err);
}

template <int NB>
static cudaError_t launch_y(const GridTable &t, cudaStream_t s) {
    const size_t sm = static_cast<size_t>(Layout<NB, uint8_t>(t.maxY).bytes);
    const cudaError_t e = ensure_dyn_smem<k_env_y<NB>>(sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_env_y<NB>, dim3(static_cast<unsigned>(t.tiles_y)), dim3(NB * 32), sm, s, t.desc, t.tmaps, t.n,
                      t.err);
}

template <int NB, int PX>
static cudaError_t launch_z(const GridTable &t, cudaStream_t s) {
    const size_t sm = static_cast<size_t>(Layout<NB, uint16_t>(t.maxZ).bytes);
    const cudaError_t e = ensure_dyn_smem<k_env_z<NB, PX>>(sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_env_z<NB, PX>, dim3(static_cast<unsigned>(t.tiles_z)), dim3(NB * 32), sm, s, t.desc, t.tmaps,
                      t.n, t.err);
}

template <int PX>
static cudaError_t launch_z_bands(const GridTable &t, int bands, cudaStream_t s) {
    switch (bands) {
        case 1: return launch_z<1, PX>(t, s);
        case 2: return launch_z<2, PX>(t, s);
        case 8: return launch_z<8, PX>(t, s);
        default: return launch_z<4, PX>(t, s);
    }
}

}  // namespace lenv

cudaError_t launch_env_y(const GridTable &t, int bands, cudaStream_t s) {
    if (t.tiles_y == 0) return cudaSuccess;
    switch (bands) {
        case 1: return lenv::launch_y<1>(t, s);
        case 2: return lenv::launch_y<2>(t, s);
        case 8: return lenv::launch_y<8>(t, s);
        default: return lenv::launch_y<4>(t, s);
    }
}

cudaError_t launch_env_z(const GridTable &t, int bands, cudaStream_t s) {
    if (t.tiles_z == 0) return cudaSuccess;
    if (t.pzx == 8) return lenv::launch_z_bands<8>(t, bands, s);
    if (t.pzx == 32) return lenv::launch_z_bands<32>(t, bands, s);
    return cudaErrorInvalidValue;   // the table's tiles were counted for another shape
}

}  // namespace vedt
