// vedt_edt_noalloc: the exact EDT of one grid without any device allocation.
//
// Some callers cannot call cudaMalloc once they are running: a hard real-time control
// loop (cudaMalloc may synchronise the whole device and has no latency bound, which can
// blow a control cycle's deadline), or a host process whose device memory is already
// reserved by another framework's allocator or capped by its environment.  For them
// this entry point keeps all EDT scratch in one fixed file-scope device array, sized for
// grids of up to kNoallocMaxVoxels padded voxels with every dimension <= 256.  Every
// GPU that loads the library holds this array until the process exits.
//
// The caller still provides the occupancy input and the two output fields.  All calls
// share the one array, which keeps whatever the last call left there; calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it and must
// be serialised by the caller.
#include <mutex>
#include <vector>

#include "vedt_internal.h"

namespace {

using namespace vedt;

constexpr int64_t kNoallocMaxVoxels = int64_t(1) << 21;    // padded X * Y * Z (128^3)
constexpr size_t kHeader = 1024;                            // GridDesc + 2 tensor maps + error word
constexpr size_t kScratchBytes = kHeader + 3 * kNoallocMaxVoxels + 256 * 256 + 1024;

// file-scope scratch: [header | xs (1 B/voxel) | s2 (2 B/voxel) | row flags | slice flags]
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_base[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per device.
// In host code g_noalloc_scratch only names a host-side stand-in, so its device address
// must come from cudaGetSymbolAddress with that device current.
cudaError_t scratch_base(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vedt_status vedt_edt_noalloc(const uint8_t *occ_dev, int32_t X, int32_t Y, int32_t Z,
                                        int32_t *sqdist_dev, int32_t *idx_dev, void *stream) {
    if (!occ_dev || !sqdist_dev || !idx_dev) return VEDT_EINVAL;
    if (X < 1 || Y < 1 || Z < 1) return VEDT_EINVAL;
    if (X > kSmallMax || Y > kSmallMax || Z > kSmallMax) return VEDT_ENOTSUP;
    const int32_t Xp = (X + kEnvCols - 1) / kEnvCols * kEnvCols;
    const int64_t Np = static_cast<int64_t>(Xp) * Y * Z;
    if (Np > kNoallocMaxVoxels) return VEDT_ENOTSUP;

    void *basev = nullptr;
    if (scratch_base(&basev) != cudaSuccess) return VEDT_ECUDA;
    uint8_t *base = static_cast<uint8_t *>(basev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // header: GridDesc at 0, tensor maps at 128 and 256, error word at 512
    GridDesc *d_desc = reinterpret_cast<GridDesc *>(base);
    CUtensorMap *d_tm = reinterpret_cast<CUtensorMap *>(base + 128);
    int32_t *d_err = reinterpret_cast<int32_t *>(base + 512);
    uint8_t *xs = base + kHeader;
    uint8_t *s2 = xs + ((Np + 255) / 256) * 256;
    uint8_t *row_has = s2 + ((2 * Np + 255) / 256) * 256;
    uint8_t *slice_has = row_has + static_cast<int64_t>(Y) * Z;

    GridDesc g{};
    g.occ = occ_dev;
    g.xs = xs;
    g.row_has = row_has;
    g.s2 = s2;
    g.slice_has = slice_has;
    g.sqdist = sqdist_dev;
    g.idx = idx_dev;
    g.X = X;
    g.Y = Y;
    g.Z = Z;
    g.Xp = Xp;
    g.row_begin = g.ty_begin = g.tz_begin = 0;
    CUtensorMap tm[2];
    const uint32_t by = static_cast<uint32_t>(Y), bz = static_cast<uint32_t>(Z);
    if (encode_tmap(&tm[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, xs, Xp, Y, Z, kEnvCols, by, 1) != CUDA_SUCCESS ||
        encode_tmap(&tm[1], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, s2, Xp, Y, Z, kEnvCols, 1, bz) != CUDA_SUCCESS)
        return VEDT_ECUDA;

    // g and tm live on this stack frame: cudaMemcpyAsync from pageable memory stages them
    // before returning, and no call below allocates device memory
    static_assert(sizeof(GridDesc) <= 128, "descriptor must fit its header slot");
    if (cudaMemcpyAsync(d_desc, &g, sizeof(GridDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_tm, tm, sizeof(tm), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(d_err, 0, sizeof(int32_t), s) != cudaSuccess)
        return VEDT_ECUDA;

    GridTable t{};
    t.desc = d_desc;
    t.tmaps = d_tm;
    t.n = 1;
    t.large = 0;
    t.maxY = Y;
    t.maxZ = Z;
    t.maxXp = Xp;
    t.rows = static_cast<int64_t>(Y) * Z;
    t.tiles_y = static_cast<int64_t>(Xp / kEnvCols) * Z;
    t.tiles_z = static_cast<int64_t>(Xp / kEnvCols) * Y;
    t.err = d_err;
    if (launch_pass_x(t, s) != cudaSuccess || launch_pass_y(t, s) != cudaSuccess ||
        launch_pass_z(t, s) != cudaSuccess)
        return VEDT_ECUDA;
    return VEDT_OK;
}
