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
// be serialised by the caller.  The grid descriptor and the two tensor maps reach the
// array as kernel parameters of a one-block header kernel (copied by the launch itself,
// so nothing refers to this call's stack once it returns).  The call waits for its
// passes and reads the device error word back, so a bounds error flagged by the
// index-checked build or an expired in-kernel wait is returned to the caller.
#include <vector>

#include "vedt_internal.h"

namespace {

using namespace vedt;

constexpr int64_t kNoallocMaxVoxels = int64_t(1) << 21;    // padded X * Y * Z (128^3)
constexpr size_t kHeader = 1024;                            // GridDesc + 2 tensor maps + error word
constexpr size_t kScratchBytes = kHeader + 3 * kNoallocMaxVoxels + 256 * 256 + 1024;

// file-scope scratch: [header | xs (1 B/voxel) | s2 (2 B/voxel) | row flags | slice flags]
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch only names a host-side stand-in, so its device address comes from
// cudaGetSymbolAddress with that device current.  It is looked up on every call (a
// runtime table lookup; the call synchronises anyway), so a module that the runtime has
// loaded again, after cudaDeviceReset or on another context, is found where it now is.
cudaError_t scratch_base(void **out) { return cudaGetSymbolAddress(out, g_noalloc_scratch); }

// The scratch header of one call: grid descriptor, the two tensor maps (64-byte aligned
// for TMA) and the cleared error word, written by thread 0 from the launch parameters.
struct NoallocHeader {
    GridDesc desc;
    alignas(64) CUtensorMap tm[2];
};

__global__ void k_noalloc_header(const __grid_constant__ NoallocHeader h, NoallocHeader *dst, int32_t *err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *dst = h;
        *err = 0;
        // the tensor maps were written through the generic proxy; release them to the
        // tensor-map proxy the passes' TMA loads read them through
        asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
    }
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
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the call ends by waiting for its own work, which a stream under capture cannot do
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return VEDT_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return VEDT_ENOTSUP;

    void *basev = nullptr;
    if (scratch_base(&basev) != cudaSuccess) return VEDT_ECUDA;
    uint8_t *base = static_cast<uint8_t *>(basev);

    // header: descriptor and tensor maps at 0, error word at 512
    static_assert(sizeof(NoallocHeader) <= 512, "header must fit its slot");
    NoallocHeader *d_hdr = reinterpret_cast<NoallocHeader *>(base);
    int32_t *d_err = reinterpret_cast<int32_t *>(base + 512);
    uint8_t *xs = base + kHeader;
    uint8_t *s2 = xs + ((Np + 255) / 256) * 256;
    uint8_t *row_has = s2 + ((2 * Np + 255) / 256) * 256;
    uint8_t *slice_has = row_has + static_cast<int64_t>(Y) * Z;

    NoallocHeader h{};
    GridDesc &g = h.desc;
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
    const uint32_t by = static_cast<uint32_t>(Y), bz = static_cast<uint32_t>(Z);
    const int px = default_pzx(&g, 1);
    if (encode_tmap(&h.tm[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, xs, Xp, Y, Z, kEnvCols, by, 1) != CUDA_SUCCESS ||
        encode_tmap(&h.tm[1], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, s2, Xp, Y, Z, static_cast<uint32_t>(px),
                    static_cast<uint32_t>(kEnvCols / px), bz) != CUDA_SUCCESS)
        return VEDT_ECUDA;
    k_noalloc_header<<<1, 32, 0, s>>>(h, d_hdr, d_err);
    if (cudaGetLastError() != cudaSuccess) return VEDT_ECUDA;

    GridTable t{};
    t.desc = &d_hdr->desc;
    t.tmaps = d_hdr->tm;
    t.n = 1;
    t.large = 0;
    t.maxY = Y;
    t.maxZ = Z;
    t.maxXp = Xp;
    t.rows = static_cast<int64_t>(Y) * Z;
    t.tiles_y = static_cast<int64_t>(Xp / kEnvCols) * Z;
    t.tiles_z = small_tiles_z(Xp, Y, px);
    t.pzx = px;
    t.err = d_err;
    if (launch_pass_x(t, s) != cudaSuccess || launch_pass_y(t, s) != cudaSuccess ||
        launch_pass_z(t, s) != cudaSuccess)
        return VEDT_ECUDA;
    // device-side errors of this call: index checks of the debug build, expired waits
    int32_t e = 0;
    if (cudaMemcpyAsync(&e, d_err, sizeof(e), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return VEDT_ECUDA;
    if (e) return (e & kErrTimeout) ? VEDT_ETIMEOUT : VEDT_ECUDA;
    return VEDT_OK;
}
