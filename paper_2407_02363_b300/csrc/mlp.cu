// Learned self-distance surrogate (not in the paper): a BF16 MLP
//   [sin q, cos q] (14) -> 4 x (Linear 256 + ReLU) -> Linear 24
// predicting the 24 per-sphere self-collision distances x_si (Eq. (selftaskvar)) that the
// exact self-map EDT produces.  Forward, backward and AdamW run in this file's kernels;
// every matrix product is a 5th-generation tensor-core GEMM:
//   C[128 x N] (+)= A[128 x K] . B[N x K]^T,   A, B bf16 K-major in shared memory,
// accumulated in fp32 in tensor memory (TMEM), issued by one thread with tcgen05.mma,
// completion signalled through tcgen05.commit on an mbarrier, read back with tcgen05.ld
// for a fused epilogue.  Operands are staged in the no-swizzle canonical K-major layout:
// 8-row x 16-byte core matrices, core matrices adjacent along K 128 bytes apart (LBO),
// adjacent along M/N (KC/8)*128 bytes apart (SBO) for a K chunk of KC elements.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "vedt_internal.h"

namespace vedt {
namespace mlpk {

using bf16 = __nv_bfloat16;

constexpr int kLayers = 5;
constexpr int kIn = 14, kOut = 24, kHidden = 256;
constexpr int kInPad = 16, kOutPad = 32;
constexpr int kThreads = 128;   // 4 warps: warp w reads TMEM lanes [32w, 32w + 32)

__host__ __device__ constexpr int layer_k(int l) { return l == 0 ? kInPad : kHidden; }
__host__ __device__ constexpr int layer_n(int l) { return l == kLayers - 1 ? kOutPad : kHidden; }
__host__ __device__ constexpr int layer_k_valid(int l) { return l == 0 ? kIn : kHidden; }
__host__ __device__ constexpr int layer_n_valid(int l) { return l == kLayers - 1 ? kOut : kHidden; }

// ---------------------------------------------------------------- tcgen05 helpers
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;   // descriptor version for tcgen05; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: fp32 accumulate, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Stages rows [r0, r0 + R) x columns [k0, k0 + KC) of a row-major bf16 matrix (row stride
// ld elements) into the canonical layout at dst: 16-byte vector v lands at dst + 16 v,
// where v = ((r / 8) * (KC / 8) + k / 8) * 8 + r % 8.  Rows >= rmax read as zero.
__device__ __forceinline__ void stage(uint8_t *dst, const bf16 *src, int ld, int r0, int rmax, int R, int k0, int KC) {
    const int kv = KC / 8;
    const int V = R * kv;
    for (int v = threadIdx.x; v < V; v += kThreads) {
        const int rr = v & 7, g = v >> 3;
        const int r = (g / kv) * 8 + rr, k8 = g % kv;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (r0 + r < rmax) val = *reinterpret_cast<const uint4 *>(src + static_cast<int64_t>(r0 + r) * ld + k0 + 8 * k8);
        *reinterpret_cast<uint4 *>(dst + 16 * v) = val;
    }
}

enum Epi { EPI_BIAS_RELU = 0, EPI_BIAS = 1, EPI_MASK = 2, EPI_ATOMIC = 3 };

struct EpiArgs {
    void *out;             // bf16 (RELU, MASK) or fp32 (BIAS, ATOMIC)
    int ldo;               // row stride of out, elements
    const float *bias;     // [N] for BIAS*, else null
    const bf16 *act;       // MASK: the layer input whose ReLU derivative gates the gradient
    int ld_act;
    int m_valid, n_valid;  // rows / columns actually stored
};

// C tile = rows [128 * blockIdx.x, +128) x all N columns; K range split over blockIdx.z
// (k_split elements each).  Block: 128 threads.
template <int N, int EPI>
__global__ void __launch_bounds__(kThreads) k_gemm(const bf16 *__restrict__ A, int lda, int rows_a,
                                                   const bf16 *__restrict__ B, int ldb, int K, int k_split,
                                                   EpiArgs ep, int32_t *err) {
    constexpr uint32_t kCols = N < 32 ? 32 : N;   // TMEM allocation: power of two >= 32
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const int kb = blockIdx.z * k_split;
    const int ke = min(K, kb + k_split);
    const int KC = ((ke - kb) % 64 == 0) ? 64 : 16;
    uint8_t *sa = smem;                            // 128 x KC
    uint8_t *sb = smem + 128 * 64 * 2;             // N x KC
    if (warp == 0) tmem_alloc(&tmem_base, kCols);
    if (tid == 0) mbar_init(&bar, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    const uint32_t idesc = idesc_bf16(128, N);
    const uint32_t sbo = static_cast<uint32_t>(KC / 8) * 128u;
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kb; k0 < ke && ok; k0 += KC) {
        stage(sa, A, lda, m0, rows_a, 128, k0, KC);
        stage(sb, B, ldb, 0, N, N, k0, KC);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int s = 0; s < KC / 16; ++s) {
                const uint64_t da = smem_desc(smem_u32(sa + s * 256), 128, sbo);
                const uint64_t db = smem_desc(smem_u32(sb + s * 256), 128, sbo);
                mma_bf16(taddr, da, db, idesc, (k0 > kb || s > 0) ? 1u : 0u);
            }
            mma_commit(&bar);
        }
        ok = mbar_wait_bounded(&bar, phase, err);
        phase ^= 1u;
        __syncthreads();
    }
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (row >= ep.m_valid) continue;
            if (EPI == EPI_ATOMIC) {
                float *o = static_cast<float *>(ep.out) + static_cast<int64_t>(row) * ep.ldo + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < ep.n_valid) atomicAdd(o + i, v[i]);
            } else if (EPI == EPI_BIAS) {
                float *o = static_cast<float *>(ep.out) + static_cast<int64_t>(row) * ep.ldo + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < ep.n_valid) o[i] = v[i] + ep.bias[c0 + i];
            } else {
                bf16 *o = static_cast<bf16 *>(ep.out) + static_cast<int64_t>(row) * ep.ldo + c0;
                alignas(16) bf16 h[16];
                if (EPI == EPI_BIAS_RELU) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(fmaxf(v[i] + ep.bias[c0 + i], 0.0f));
                } else {
                    const bf16 *a = ep.act + static_cast<int64_t>(row) * ep.ld_act + c0;
                    alignas(16) bf16 av[16];
                    *reinterpret_cast<uint4 *>(av) = *reinterpret_cast<const uint4 *>(a);
                    *reinterpret_cast<uint4 *>(av + 8) = *reinterpret_cast<const uint4 *>(a + 8);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        h[i] = __float2bfloat16_rn(__bfloat162float(av[i]) > 0.0f ? v[i] : 0.0f);
                }
                *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(h + 8);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, kCols);
}

// ---------------------------------------------------------------- small kernels
// features [sin q, cos q, 0, 0] as bf16, rows >= B zero
__global__ void k_features(const float *__restrict__ q, int B, int rows, bf16 *__restrict__ x) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(rows) * kInPad) return;
    const int b = static_cast<int>(t / kInPad), j = static_cast<int>(t % kInPad);
    float v = 0.0f;
    if (b < B && j < kIn) v = j < 7 ? sinf(q[b * 7 + j]) : cosf(q[b * 7 + j - 7]);
    x[t] = __float2bfloat16_rn(v);
}

// out [rows][kOutPad] fp32 -> user [B][24]
__global__ void k_copy_out(const float *__restrict__ o, int B, float *__restrict__ user) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * kOut) return;
    user[t] = o[(t / kOut) * kOutPad + t % kOut];
}

// sums[0] += sum (diff^2), sums[1] += sum mask  over b < B, i < 24
__global__ void k_loss_sums(const float *__restrict__ o, const float *__restrict__ y, const float *__restrict__ mask,
                            int B, float *sums) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f, mc = 0.f;
    if (t < B * kOut) {
        const float m = mask ? mask[t] : 1.0f;
        const float d = (o[(t / kOut) * kOutPad + t % kOut] - y[t]) * m;
        d2 = d * d;
        mc = m;
    }
    for (int s = 16; s > 0; s >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, s);
        mc += __shfl_down_sync(0xffffffffu, mc, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(sums, d2);
        atomicAdd(sums + 1, mc);
    }
}

// dL/dout = 2 (out - y) mask / count  as bf16 [rows][kOutPad]
__global__ void k_loss_grad(const float *__restrict__ o, const float *__restrict__ y, const float *__restrict__ mask,
                            int B, int rows, const float *__restrict__ sums, bf16 *__restrict__ g) {
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(rows) * kOutPad) return;
    const int b = static_cast<int>(t / kOutPad), i = static_cast<int>(t % kOutPad);
    float v = 0.f;
    if (b < B && i < kOut) {
        const int u = b * kOut + i;
        const float m = mask ? mask[u] : 1.0f;
        v = 2.0f * (o[t] - y[u]) * m / fmaxf(sums[1], 1.0f);
    }
    g[t] = __float2bfloat16_rn(v);
}

// out[c][r] = in[r][c] for r < R, c < C; out has row stride ldo; rows c in [C, Cpad) zero
__global__ void k_transpose(const bf16 *__restrict__ in, int R, int C, int ldi, bf16 *__restrict__ out, int Cpad,
                            int ldo) {
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < R && c < C) ? in[static_cast<int64_t>(r) * ldi + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < Cpad && r < R) out[static_cast<int64_t>(c) * ldo + r] = tile[threadIdx.x][i];
    }
}

// db[n] = sum_b g[b][n]
__global__ void k_bias_grad(const bf16 *__restrict__ g, int B, int N, int ld, float *__restrict__ db) {
    const int n = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += __bfloat162float(g[static_cast<int64_t>(b) * ld + n]);
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < (blockDim.x + 31) / 32; ++i) t += part[i];
        db[n] = t;
    }
}

// AdamW on the padded flat parameters (padding stays zero: its gradient is zero)
__global__ void k_adamw(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                        float *__restrict__ v, int64_t n, float lr, float wd, float b1, float b2, float eps,
                        float c1, float c2) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
}

// bf16 copies of one layer's weights: W [N][K] and W^T [K][N]
__global__ void k_to_bf16(const float *__restrict__ w, int N, int K, bf16 *__restrict__ wb, bf16 *__restrict__ wt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * K) return;
    const int n = t / K, k = t % K;
    const bf16 h = __float2bfloat16_rn(w[t]);
    wb[t] = h;
    wt[k * N + n] = h;
}

// ---------------------------------------------------------------- fused forward
// All five layers run in one persistent kernel, one CTA per SM.  A CTA holds two 128-row
// tiles ("slots") at once: each slot has its activation tile (128 x 256 bf16, canonical
// K-major layout, SBO 4096 B) in shared memory and its own 256-column fp32 accumulator
// in tensor memory (the two fill all 512 columns).  Warp roles:
//   warp 0, lane 0   streams weight chunks into a ring of kStages shared-memory stages
//                    with bulk asynchronous copies (cp.async.bulk, mbarrier completion),
//                    in the order the MMA thread consumes them;
//   warp 1, lane 0   issues the tcgen05.mma: every weight chunk feeds both slots;
//   warps 2..9       epilogue of slot 0, warps 10..17 of slot 1 (two warps per TMEM lane
//                    quadrant, one per column half): read the finished accumulator from
//                    tensor memory, add bias, ReLU, round to bf16 and write the next
//                    layer's input in place (or the fp32 output after the last layer),
//                    then start the slot's next tile with its features.
// Weight bytes, not MMAs, set the pace when a chunk feeds only 128 rows: a 32 KB chunk
// holds 4 MMAs of work per slot, and a ring of three stages then buffers less tensor work
// than one copy round trip lasts.  Feeding both slots from each chunk doubles the work per
// byte; the price is that a layer's epilogue cannot overlap the same layer's MMAs, so the
// MMA thread orders its work to hide most of it: slot 0's accumulator is committed before
// slot 1's last MMAs, and at the next layer slot 1 waits behind slot 0's first chunk.
// The weights are read as 14 pre-packed chunk images (each the exact shared-memory image
// of its K columns), written by k_pack_w whenever the parameters change.
struct WChunk {
    int l, k0, kc, n, off;   // layer, first K column, K width, N rows, byte offset in the image
};
constexpr int kWKC = 64;                                  // K width of hidden-layer chunks
constexpr int kChunksPerHidden = kHidden / kWKC;          // 4
constexpr int kNumWChunks = 1 + 3 * kChunksPerHidden + 1; // 14
constexpr int kStageBytes = kHidden * kWKC * 2;           // 32 KB
constexpr int kWImageBytes = kHidden * kInPad * 2 + 3 * kChunksPerHidden * kStageBytes + kOutPad * kHidden * 2;

__host__ __device__ constexpr WChunk wchunk(int c) {
    return c == 0 ? WChunk{0, 0, kInPad, kHidden, 0}
           : c <= 3 * kChunksPerHidden
               ? WChunk{1 + (c - 1) / kChunksPerHidden, ((c - 1) % kChunksPerHidden) * kWKC, kWKC, kHidden,
                        kHidden * kInPad * 2 + (c - 1) * kStageBytes}
               : WChunk{kLayers - 1, 0, kHidden, kOutPad, kHidden * kInPad * 2 + 3 * kChunksPerHidden * kStageBytes};
}
// first chunk of layer l (l = kLayers gives the end)
__host__ __device__ constexpr int layer_chunk_begin(int l) {
    return l == 0 ? 0 : (l < kLayers ? 1 + (l - 1) * kChunksPerHidden : kNumWChunks);
}
static_assert(wchunk(kNumWChunks - 1).off + kOutPad * kHidden * 2 == kWImageBytes, "weight image size");

// The order a CTA consumes a tile pair's chunks in: a hidden layer's four K chunks start
// at chunk `rot` of the layer (CTA index mod 4; the accumulation order does not matter to
// the result beyond fp32 rounding), so at any time the CTAs read four different chunks and
// the L2 lines of one chunk are not requested by every SM at once.
__host__ __device__ constexpr int chunk_order(int p, int rot) {
    return (p == 0 || p == kNumWChunks - 1)
               ? p
               : 1 + ((p - 1) / kChunksPerHidden) * kChunksPerHidden + ((p - 1) % kChunksPerHidden + rot) % kChunksPerHidden;
}

// packs the bf16 weights W_l [N_l][K_l] into the chunk images
__global__ void k_pack_w(const bf16 *w0, const bf16 *w1, const bf16 *w2, const bf16 *w3, const bf16 *w4,
                         uint8_t *__restrict__ img) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kWImageBytes / 16) return;
    int c = 0;
    while (c + 1 < kNumWChunks && wchunk(c + 1).off <= 16 * t) ++c;
    const WChunk ch = wchunk(c);
    const int v = t - ch.off / 16;
    const int kv = ch.kc / 8, rr = v & 7, g = v >> 3;
    const int r = (g / kv) * 8 + rr, k8 = g % kv;
    const bf16 *W = ch.l == 0 ? w0 : ch.l == 1 ? w1 : ch.l == 2 ? w2 : ch.l == 3 ? w3 : w4;
    *reinterpret_cast<uint4 *>(img + 16 * static_cast<int64_t>(t)) =
        *reinterpret_cast<const uint4 *>(W + static_cast<int64_t>(r) * layer_k(ch.l) + ch.k0 + 8 * k8);
}

// Passed by value and read in place (__grid_constant__): the biases sit in the constant
// bank, whose cache broadcasts the one column value a warp's lanes read together; with
// the SM's shared memory taken by tiles and weights, L1 loads of them stall the epilogue.
struct FusedArgs {
    const uint8_t *wimg;                  // packed weight chunk images
    float bias[kLayers - 1][kHidden];     // hidden-layer biases
    float bias_out[kOutPad];              // output-layer bias (first kOut used)
};

constexpr int kStages = 3;
constexpr int kActBytes = 128 * kHidden * 2;               // 64 KB per slot
constexpr int kFusedThreads = 64 + 16 * 32;   // producer, MMA, 2 x 8 epilogue warps
constexpr int kFusedSmem = 2 * kActBytes + kStages * kStageBytes;   // 224 KB

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// two fp32 values -> packed bf16 pair (x in the low half), round to nearest even, negatives to 0
__device__ __forceinline__ uint32_t relu_bf16x2(float x, float y) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(y), "f"(x));
    return d;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 64 consecutive columns of the warp's 32 lanes, waited for inside the same statement (so
// no use of r can be scheduled before the load completes)
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
}

// two fp32 values -> packed bf16 pair (x in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(y), "f"(x));
    return d;
}

// features [sin q, cos q, 0, 0] of one row as bf16, in the order of the layer-0 input
struct Feat {
    uint4 lo, hi;
};
__device__ __forceinline__ Feat features_of(int row, const float *q, int B) {
    float sn[7], cs[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        const float x = row < B ? q[static_cast<int64_t>(row) * 7 + j] : 0.f;
        sn[j] = row < B ? sinf(x) : 0.f;
        cs[j] = row < B ? cosf(x) : 0.f;
    }
    Feat f;
    f.lo = make_uint4(pack_bf16x2(sn[0], sn[1]), pack_bf16x2(sn[2], sn[3]), pack_bf16x2(sn[4], sn[5]),
                      pack_bf16x2(sn[6], cs[0]));
    f.hi = make_uint4(pack_bf16x2(cs[1], cs[2]), pack_bf16x2(cs[3], cs[4]), pack_bf16x2(cs[5], cs[6]), 0u);
    return f;
}
// row rl of a slot's layer-0 input tile (K = 16 layout, SBO 256 B)
__device__ __forceinline__ void store_features(uint8_t *act, int rl, const Feat &f) {
    const int base = (rl >> 3) * 256 + (rl & 7) * 16;
    *reinterpret_cast<uint4 *>(act + base) = f.lo;
    *reinterpret_cast<uint4 *>(act + base + 128) = f.hi;
}

// Local tile i of this CTA is global tile blockIdx.x + i * gridDim.x and lives in slot
// i & 1; local pair p holds tiles 2p and 2p + 1 (the last pair may hold one).  Rows past
// the batch compute on zero features and store nothing.
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_mlp_fused(const float *__restrict__ q, int B, const __grid_constant__ FusedArgs a, float *__restrict__ out,
                int32_t *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t full[kStages], empty[kStages], acc_full[2], act_ready[2], fin;
    __shared__ uint32_t tmem_base;
    uint8_t *stage = smem + 2 * kActBytes;    // activation tile of slot s at smem + s * kActBytes
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rot = static_cast<int>(blockIdx.x) % kChunksPerHidden;   // see chunk_order
    const int n_tiles = (B + 127) / 128;
    const int T = static_cast<int>(blockIdx.x) < n_tiles ? (n_tiles - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
    const int pairs = (T + 1) / 2;
    auto tile_row0 = [&](int i) { return (static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x)) * 128; };
    // A forward launched right after another starts placing its CTAs as the previous grid's
    // leave their SMs; everything up to the dependency wait below touches only on-chip
    // state (tensor memory, shared-memory barriers; the biases are launch parameters).
    pdl_trigger();
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    if (tid == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&act_ready[s], 8);        // one arrival per epilogue warp of the slot
        }
        mbar_init(&fin, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    pdl_wait();   // weights, joint angles and outputs may belong to the previous kernels

    if (warp == 0 && lane == 0) {
        // ---- weight producer: one thread fills the ring in consumption order (chunk it goes
        // to stage it mod kStages once the chunk kStages before it is consumed).  One thread,
        // not one lane per stage: lanes of a warp spinning on different barriers take turns,
        // and a stage whose barrier completed waits for another lane's spin.
        const uint32_t total = static_cast<uint32_t>(pairs * kNumWChunks);
        bool ok = true;
        uint32_t it = 0;
        for (; it < total && ok; ++it) {
            const uint32_t k = it % kStages;
            if (it >= kStages && !(ok = mbar_wait_bounded(&empty[k], ((it / kStages) - 1) & 1, err))) break;
            const WChunk ch = wchunk(chunk_order(static_cast<int>(it % kNumWChunks), rot));
            const uint32_t bytes = static_cast<uint32_t>(ch.n * ch.kc * 2);
            mbar_arrive_expect_tx(&full[k], bytes);
            bulk_load(stage + k * kStageBytes, a.wimg + ch.off, bytes, &full[k]);
        }
        // the last copy into each stage has landed before the CTA exits (normally consumed)
        for (uint32_t j = it > kStages ? it - kStages : 0; j < it; ++j)
            mbar_wait_bounded(&full[j % kStages], (j / kStages) & 1, err);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer.  The tensor pipe idles whenever this thread spends time between
        // MMAs, so descriptors are built once per layer and advanced by constants (the start
        // address field counts 16-byte units), and the ring index advances without division.
        const uint32_t id256 = idesc_bf16(128, kHidden), id32 = idesc_bf16(128, kOutPad);
        const uint32_t stage0 = smem_u32(stage);
        constexpr uint64_t kStageStep = kStageBytes >> 4;
        constexpr uint64_t kSlotStep = kActBytes >> 4;
        const uint64_t a_l0 = smem_desc(smem_u32(smem), 128, 256), a_h = smem_desc(smem_u32(smem), 128, (kHidden / 8) * 128);
        const uint64_t b_l0 = smem_desc(stage0, 128, 256), b_h = smem_desc(stage0, 128, (kWKC / 8) * 128),
                       b_out = smem_desc(stage0, 128, (kHidden / 8) * 128);
        uint32_t k = 0, phase = 0, ready0 = 0, ready1 = 0;
        bool ok = true;
        auto next_stage = [&]() {
            if (++k == kStages) {
                k = 0;
                phase ^= 1u;
            }
        };
        auto wait_full = [&]() {
            ok = mbar_wait_bounded(&full[k], phase, err);
            tc_fence_after();
            return ok;
        };
        auto wait_ready = [&](int s) {
            ok = mbar_wait_bounded(&act_ready[s], (s ? ready1++ : ready0++) & 1, err);
            tc_fence_after();
            return ok;
        };
        for (int p = 0; p < pairs && ok; ++p) {
            const int ns = (2 * p + 1 < T) ? 2 : 1;
            for (int l = 0; l < kLayers && ok; ++l) {
                if (l == 0) {                           // K = 16: one MMA per slot
                    if (!wait_full()) break;
                    for (int s = 0; s < ns; ++s) {
                        if (!wait_ready(s)) break;
                        mma_bf16(taddr + s * 256, a_l0 + s * kSlotStep, b_l0 + k * kStageStep, id256, 0u);
                        mma_commit(&acc_full[s]);
                    }
                    if (!ok) break;
                    mma_commit(&empty[k]);
                    next_stage();
                } else if (l < kLayers - 1) {           // four chunks of K = 64, four MMAs per slot each
                    for (int c = 0; c < kChunksPerHidden; ++c) {
                        if (!wait_full()) break;
                        const uint64_t b0 = b_h + k * kStageStep;
                        const int cr = (c + rot) % kChunksPerHidden;   // the K chunk this stage holds
                        for (int s = 0; s < ns; ++s) {
                            if (c == 0 && !wait_ready(s)) break;
                            const uint64_t a0 = a_h + s * kSlotStep + static_cast<uint64_t>(cr * (kWKC / 16) * 16);
                            const uint32_t d = taddr + s * 256;
#pragma unroll
                            for (int st = 0; st < kWKC / 16; ++st)
                                mma_bf16(d, a0 + st * 16, b0 + st * 16, id256, (c | st) ? 1u : 0u);
                            if (c == kChunksPerHidden - 1) mma_commit(&acc_full[s]);
                        }
                        if (!ok) break;
                        mma_commit(&empty[k]);
                        next_stage();
                    }
                } else {                                // N = 32, K = 256 in one chunk
                    if (!wait_full()) break;
                    const uint64_t b0 = b_out + k * kStageStep;
                    for (int s = 0; s < ns; ++s) {
                        if (!wait_ready(s)) break;
                        const uint32_t d = taddr + s * 256;
#pragma unroll
                        for (int st = 0; st < kHidden / 16; ++st)
                            mma_bf16(d, a_h + s * kSlotStep + st * 16, b0 + st * 16, id32, st ? 1u : 0u);
                        mma_commit(&acc_full[s]);
                    }
                    if (!ok) break;
                    mma_commit(&empty[k]);
                    next_stage();
                }
            }
        }
        // all MMAs issued by this thread have completed before tensor memory is released
        mma_commit(&fin);
        mbar_wait_bounded(&fin, 0, err);
    } else if (warp >= 2) {
        // ---- epilogue.  Warps 2..9 serve slot 0 and 10..17 slot 1; in a slot, warps e and
        // e + 4 share TMEM lane quadrant warp % 4 and take the lower / upper 128 columns.
        // At the output layer the lower half stores the outputs while the upper half stores
        // the slot's next tile's features, computed after the layer-1 epilogue while the
        // layer-2 MMAs run (their global loads and sin / cos stay off the layer boundaries).
        const int e = warp - 2;
        const int s = e >> 3, half = (e >> 2) & 1, quad = warp & 3;
        const int rl = quad * 32 + lane;
        const uint32_t tq = taddr + (static_cast<uint32_t>(quad * 32) << 16) + s * 256 + half * 128;
        uint8_t *my_act = smem + s * kActBytes;
        const bool vec_out = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
        // a warp's lanes publish their shared-memory writes to the tensor cores' (async)
        // proxy, the warp converges (ordering the lanes' writes before lane 0), and lane 0
        // arrives for the warp
        auto release = [&]() {
            tc_fence_before();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&act_ready[s]);
        };
        // The layer loop is unrolled and the column half is a compile-time constant, so
        // every bias is a fixed offset into the kernel's constant bank (an FADD operand,
        // no load instruction).
        auto run = [&](auto half_c) {
            constexpr int HALF = decltype(half_c)::value;
            Feat f{};
            if (s < T) {
                if (HALF) store_features(my_act, rl, features_of(tile_row0(s) + rl, q, B));
                release();
            }
            uint32_t accn = 0;
            bool ok = true;
            for (int i = s; i < T && ok; i += 2) {
#pragma unroll
                for (int l = 0; l < kLayers; ++l) {
                    if (!(ok = mbar_wait_bounded(&acc_full[s], accn++ & 1, err))) break;
                    tc_fence_after();
                    if (l < kLayers - 1) {
#pragma unroll
                        for (int c0 = 0; c0 < 128; c0 += 64) {
                            uint32_t r[64];
                            tmem_ld64(tq + c0, r);
#pragma unroll
                            for (int h = 0; h < 8; ++h) {
                                const int col = HALF * 128 + c0 + 8 * h;
                                const float *bc = a.bias[l] + col;
                                uint4 o;
                                o.x = relu_bf16x2(__uint_as_float(r[8 * h + 0]) + bc[0], __uint_as_float(r[8 * h + 1]) + bc[1]);
                                o.y = relu_bf16x2(__uint_as_float(r[8 * h + 2]) + bc[2], __uint_as_float(r[8 * h + 3]) + bc[3]);
                                o.z = relu_bf16x2(__uint_as_float(r[8 * h + 4]) + bc[4], __uint_as_float(r[8 * h + 5]) + bc[5]);
                                o.w = relu_bf16x2(__uint_as_float(r[8 * h + 6]) + bc[6], __uint_as_float(r[8 * h + 7]) + bc[7]);
                                const int base = ((rl >> 3) * (kHidden / 8) + (col >> 3)) * 128 + (rl & 7) * 16;
                                *reinterpret_cast<uint4 *>(my_act + base) = o;
                            }
                        }
                    } else {
                        if (!HALF) {
                            uint32_t r[32];
                            tmem_ld32(tq, r);
                            const int row = tile_row0(i) + rl;
                            float v[kOut];
#pragma unroll
                            for (int j = 0; j < kOut; ++j) v[j] = __uint_as_float(r[j]) + a.bias_out[j];
                            if (row < B) {
                                float *o = out + static_cast<int64_t>(row) * kOut;
                                if (vec_out) {
#pragma unroll
                                    for (int j = 0; j < kOut / 4; ++j)
                                        reinterpret_cast<float4 *>(o)[j] =
                                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                                } else {
#pragma unroll
                                    for (int j = 0; j < kOut; ++j) o[j] = v[j];
                                }
                            }
                        }
                        if (i + 2 >= T) break;   // this slot has no further tile
                        if (HALF) store_features(my_act, rl, f);
                    }
                    release();
                    // the slot's next tile's features, for its output-layer epilogue: computed
                    // while this tile's layer-2 MMAs run, off the layer boundaries
                    if (l == 1 && HALF && i + 2 < T) f = features_of(tile_row0(i + 2) + rl, q, B);
                }
            }
        };
        if (half)
            run(std::integral_constant<int, 1>{});
        else
            run(std::integral_constant<int, 0>{});
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(taddr, 512);
    }
}

}  // namespace mlpk
}  // namespace vedt

using namespace vedt;
using namespace vedt::mlpk;

struct vedt_mlp {
    int cap = 0;                 // batch capacity, multiple of 128
    cudaStream_t stream = nullptr;
    int64_t np = 0;              // padded parameter count
    int64_t offW[kLayers], offB[kLayers];
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // fp32 padded
    bf16 *wb[kLayers] = {}, *wt[kLayers] = {};
    uint8_t *wimg = nullptr;     // packed weight chunk images of the fused forward
    FusedArgs fused{};           // fused-forward arguments, biases copied from p
    bool fused_valid = false;    // fused.bias matches the device parameters
    int sms = 1;                 // SM count
    bf16 *x0 = nullptr;          // [cap][16]
    bf16 *act[kLayers - 1] = {}; // [cap][256]
    float *out = nullptr;        // [cap][32]
    bf16 *dz[2] = {};            // [cap][256]
    bf16 *tA = nullptr, *tB = nullptr;   // [256][cap] transposes
    float *sums = nullptr;       // loss sums (2)
    int32_t *err = nullptr;
    int64_t step = 0;
};

namespace {

vedt_status from_cuda(cudaError_t e) {
    return e == cudaSuccess ? VEDT_OK : (e == cudaErrorMemoryAllocation ? VEDT_ENOMEM : VEDT_ECUDA);
}

#define MCHECK(call)                                 \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

template <int N, int EPI>
cudaError_t gemm(const bf16 *A, int lda, int rows_a, int M, const bf16 *B, int ldb, int K, int k_split,
                 const EpiArgs &ep, int32_t *err, cudaStream_t s) {
    const size_t smem = 128 * 64 * 2 + static_cast<size_t>(N) * 64 * 2;
    cudaError_t e = ensure_dyn_smem<k_gemm<N, EPI>>(smem);
    if (e != cudaSuccess) return e;
    const int splits = (K + k_split - 1) / k_split;
    dim3 grid((M + 127) / 128, 1, splits);
    k_gemm<N, EPI><<<grid, kThreads, smem, s>>>(A, lda, rows_a, B, ldb, K, k_split, ep, err);
    return cudaGetLastError();
}

// forward through all layers for `rows` rows (multiple of 128) of x0
vedt_status forward_rows(vedt_mlp *n, int rows) {
    cudaStream_t s = n->stream;
    const bf16 *in = n->x0;
    for (int l = 0; l < kLayers; ++l) {
        EpiArgs ep{};
        ep.bias = n->p + n->offB[l];
        ep.m_valid = rows;
        if (l < kLayers - 1) {
            ep.out = n->act[l];
            ep.ldo = kHidden;
            ep.n_valid = kHidden;
            MCHECK((gemm<kHidden, EPI_BIAS_RELU>(in, layer_k(l), rows, rows, n->wb[l], layer_k(l), layer_k(l),
                                                 layer_k(l), ep, n->err, s)));
            in = n->act[l];
        } else {
            ep.out = n->out;
            ep.ldo = kOutPad;
            ep.n_valid = kOutPad;
            MCHECK((gemm<kOutPad, EPI_BIAS>(in, kHidden, rows, rows, n->wb[l], kHidden, kHidden, kHidden, ep, n->err,
                                            s)));
        }
    }
    return VEDT_OK;
}

vedt_status features(vedt_mlp *n, const float *q, int B, int rows) {
    const int64_t tot = static_cast<int64_t>(rows) * kInPad;
    k_features<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, n->stream>>>(q, B, rows, n->x0);
    MCHECK(cudaGetLastError());
    return VEDT_OK;
}

vedt_status refresh_bf16(vedt_mlp *n) {
    for (int l = 0; l < kLayers; ++l) {
        const int N = layer_n(l), K = layer_k(l);
        k_to_bf16<<<(N * K + 255) / 256, 256, 0, n->stream>>>(n->p + n->offW[l], N, K, n->wb[l], n->wt[l]);
        MCHECK(cudaGetLastError());
    }
    k_pack_w<<<(kWImageBytes / 16 + 255) / 256, 256, 0, n->stream>>>(n->wb[0], n->wb[1], n->wb[2], n->wb[3], n->wb[4],
                                                                     n->wimg);
    MCHECK(cudaGetLastError());
    return VEDT_OK;
}

// loss sums, output gradient and backward pass into n->g (padded layout)
vedt_status backward(vedt_mlp *n, const float *y, const float *mask, int B, int rows) {
    cudaStream_t s = n->stream;
    MCHECK(cudaMemsetAsync(n->sums, 0, 2 * sizeof(float), s));
    k_loss_sums<<<(B * kOut + 255) / 256, 256, 0, s>>>(n->out, y, mask, B, n->sums);
    MCHECK(cudaGetLastError());
    bf16 *dcur = n->dz[0], *dnext = n->dz[1];
    {
        const int64_t tot = static_cast<int64_t>(rows) * kOutPad;
        k_loss_grad<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(n->out, y, mask, B, rows, n->sums, dcur);
        MCHECK(cudaGetLastError());
    }
    MCHECK(cudaMemsetAsync(n->g, 0, sizeof(float) * n->np, s));
    for (int l = kLayers - 1; l >= 0; --l) {
        const int N = layer_n(l), K = layer_k(l);
        const bf16 *ain = l == 0 ? n->x0 : n->act[l - 1];
        // dW_l = dZ_l^T . A_(l-1): M = N (rows padded to 128), N_gemm = K, K_gemm = rows
        {
            dim3 tb(32, 8);
            k_transpose<<<dim3((rows + 31) / 32, (std::max(N, 128) + 31) / 32), tb, 0, s>>>(
                dcur, rows, N, N, n->tA, std::max(N, 128), rows);
            MCHECK(cudaGetLastError());
            k_transpose<<<dim3((rows + 31) / 32, (K + 31) / 32), tb, 0, s>>>(ain, rows, K, K, n->tB, K, rows);
            MCHECK(cudaGetLastError());
            EpiArgs ep{};
            ep.out = n->g + n->offW[l];
            ep.ldo = K;
            ep.m_valid = N;
            ep.n_valid = K;
            const int ks = rows >= 1024 ? 1024 : rows;
            if (K == kHidden)
                MCHECK((gemm<kHidden, EPI_ATOMIC>(n->tA, rows, std::max(N, 128), std::max(N, 128), n->tB, rows, rows,
                                                  ks, ep, n->err, s)));
            else
                MCHECK((gemm<kInPad, EPI_ATOMIC>(n->tA, rows, std::max(N, 128), std::max(N, 128), n->tB, rows, rows,
                                                 ks, ep, n->err, s)));
        }
        k_bias_grad<<<N, 256, 0, s>>>(dcur, B, N, N, n->g + n->offB[l]);
        MCHECK(cudaGetLastError());
        if (l > 0) {
            // dZ_(l-1) = (dZ_l . W_l) * (A_(l-1) > 0): M = rows, N_gemm = K, K_gemm = N
            EpiArgs ep{};
            ep.out = dnext;
            ep.ldo = K;
            ep.act = n->act[l - 1];
            ep.ld_act = K;
            ep.m_valid = rows;
            ep.n_valid = K;
            MCHECK((gemm<kHidden, EPI_MASK>(dcur, N, rows, rows, n->wt[l], N, N, N, ep, n->err, s)));
            std::swap(dcur, dnext);
        }
    }
    return VEDT_OK;
}

void free_mlp(vedt_mlp *n) {
    cudaFree(n->p);
    cudaFree(n->g);
    cudaFree(n->m);
    cudaFree(n->v);
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(n->wb[l]);
        cudaFree(n->wt[l]);
    }
    cudaFree(n->wimg);
    cudaFree(n->x0);
    for (int l = 0; l < kLayers - 1; ++l) cudaFree(n->act[l]);
    cudaFree(n->out);
    cudaFree(n->dz[0]);
    cudaFree(n->dz[1]);
    cudaFree(n->tA);
    cudaFree(n->tB);
    cudaFree(n->sums);
    cudaFree(n->err);
    delete n;
}

bool check_rows(const vedt_mlp *n, int B) { return n && B >= 1 && B <= n->cap; }

// persistent grid: one CTA per SM, capped by the number of 128-row tiles
cudaError_t launch_fused(const vedt_mlp *n, const float *q, int B, const FusedArgs &a, float *out) {
    const int tiles = (B + 127) / 128;
    return launch_pdl(k_mlp_fused, dim3(std::min(tiles, n->sms)), dim3(kFusedThreads), kFusedSmem, n->stream, q, B,
                      a, out, n->err);
}

}  // namespace

extern "C" {

vedt_status vedt_mlp_create(int batch_capacity, void *stream, vedt_mlp **out) {
    if (!out || batch_capacity < 1 || batch_capacity > (1 << 22)) return VEDT_EINVAL;
    *out = nullptr;
    vedt_mlp *n = new (std::nothrow) vedt_mlp();
    if (!n) return VEDT_ENOMEM;
    n->cap = (batch_capacity + 127) / 128 * 128;
    n->stream = static_cast<cudaStream_t>(stream);
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->offW[l] = off;
        off += static_cast<int64_t>(layer_n(l)) * layer_k(l);
        n->offB[l] = off;
        off += layer_n(l);
    }
    n->np = off;
    const int64_t cap = n->cap;
    cudaError_t e = cudaSuccess;
    for (float **pp : {&n->p, &n->g, &n->m, &n->v})
        if (e == cudaSuccess) e = cudaMalloc(pp, sizeof(float) * n->np);
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        e = cudaMalloc(&n->wb[l], sizeof(bf16) * layer_n(l) * layer_k(l));
        if (e == cudaSuccess) e = cudaMalloc(&n->wt[l], sizeof(bf16) * layer_n(l) * layer_k(l));
    }
    if (e == cudaSuccess) e = cudaMalloc(&n->wimg, kWImageBytes);
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem);
    if (e == cudaSuccess) e = cudaMalloc(&n->x0, sizeof(bf16) * cap * kInPad);
    for (int l = 0; l < kLayers - 1 && e == cudaSuccess; ++l) e = cudaMalloc(&n->act[l], sizeof(bf16) * cap * kHidden);
    if (e == cudaSuccess) e = cudaMalloc(&n->out, sizeof(float) * cap * kOutPad);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&n->dz[i], sizeof(bf16) * cap * kHidden);
    if (e == cudaSuccess) e = cudaMalloc(&n->tA, sizeof(bf16) * cap * kHidden);
    if (e == cudaSuccess) e = cudaMalloc(&n->tB, sizeof(bf16) * cap * kHidden);
    if (e == cudaSuccess) e = cudaMalloc(&n->sums, sizeof(float) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int32_t));
    for (float *pp : {n->p, n->g, n->m, n->v})
        if (e == cudaSuccess) e = cudaMemset(pp, 0, sizeof(float) * n->np);
    if (e != cudaSuccess) {
        free_mlp(n);
        return from_cuda(e);
    }
    *out = n;
    return VEDT_OK;
}

vedt_status vedt_mlp_destroy(vedt_mlp *n) {
    if (!n) return VEDT_OK;
    cudaStreamSynchronize(n->stream);
    free_mlp(n);
    return VEDT_OK;
}

int64_t vedt_mlp_num_params(void) {
    int64_t c = 0;
    for (int l = 0; l < kLayers; ++l) c += static_cast<int64_t>(layer_n_valid(l)) * layer_k_valid(l) + layer_n_valid(l);
    return c;
}

// flat host layout -> the padded device layout (zeros in the padding)
static std::vector<float> padded(const vedt_mlp *n, const float *flat) {
    std::vector<float> pad(static_cast<size_t>(n->np), 0.f);
    int64_t r = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int Nv = layer_n_valid(l), Kv = layer_k_valid(l), K = layer_k(l);
        for (int i = 0; i < Nv; ++i)
            for (int k = 0; k < Kv; ++k) pad[n->offW[l] + static_cast<int64_t>(i) * K + k] = flat[r++];
        for (int i = 0; i < Nv; ++i) pad[n->offB[l] + i] = flat[r++];
    }
    return pad;
}

vedt_status vedt_mlp_set_params(vedt_mlp *n, const float *params, int64_t count) {
    if (!n || !params || count != vedt_mlp_num_params()) return VEDT_EINVAL;
    const std::vector<float> pad = padded(n, params);
    MCHECK(cudaMemcpyAsync(n->p, pad.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice, n->stream));
    MCHECK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->stream));
    MCHECK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->stream));
    n->step = 0;
    n->fused_valid = false;
    vedt_status st = refresh_bf16(n);
    if (st != VEDT_OK) return st;
    MCHECK(cudaStreamSynchronize(n->stream));
    return VEDT_OK;
}

static vedt_status unpad(vedt_mlp *n, const float *dev, float *host, int64_t count) {
    if (count != vedt_mlp_num_params()) return VEDT_EINVAL;
    std::vector<float> pad(static_cast<size_t>(n->np));
    MCHECK(cudaMemcpyAsync(pad.data(), dev, sizeof(float) * n->np, cudaMemcpyDeviceToHost, n->stream));
    MCHECK(cudaStreamSynchronize(n->stream));
    int64_t r = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int Nv = layer_n_valid(l), Kv = layer_k_valid(l), K = layer_k(l);
        for (int i = 0; i < Nv; ++i)
            for (int k = 0; k < Kv; ++k) host[r++] = pad[n->offW[l] + static_cast<int64_t>(i) * K + k];
        for (int i = 0; i < Nv; ++i) host[r++] = pad[n->offB[l] + i];
    }
    return VEDT_OK;
}

vedt_status vedt_mlp_get_params(vedt_mlp *n, float *params, int64_t count) {
    if (!n || !params) return VEDT_EINVAL;
    return unpad(n, n->p, params, count);
}

vedt_status vedt_mlp_get_state(vedt_mlp *n, float *params, float *m1, float *m2, int64_t count, int64_t *step) {
    if (!n || !params || !m1 || !m2 || !step) return VEDT_EINVAL;
    vedt_status st = unpad(n, n->p, params, count);
    if (st == VEDT_OK) st = unpad(n, n->m, m1, count);
    if (st == VEDT_OK) st = unpad(n, n->v, m2, count);
    if (st == VEDT_OK) *step = n->step;
    return st;
}

vedt_status vedt_mlp_set_state(vedt_mlp *n, const float *params, const float *m1, const float *m2, int64_t count,
                               int64_t step) {
    if (!n || !params || !m1 || !m2 || step < 0 || count != vedt_mlp_num_params()) return VEDT_EINVAL;
    vedt_status st = vedt_mlp_set_params(n, params, count);   // also refreshes the bf16 copies
    if (st != VEDT_OK) return st;
    const std::vector<float> a = padded(n, m1), b = padded(n, m2);
    MCHECK(cudaMemcpyAsync(n->m, a.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice, n->stream));
    MCHECK(cudaMemcpyAsync(n->v, b.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice, n->stream));
    MCHECK(cudaStreamSynchronize(n->stream));
    n->step = step;
    return VEDT_OK;
}

vedt_status vedt_mlp_forward(vedt_mlp *n, const float *q_dev, int B, float *out_dev) {
    if (!check_rows(n, B) || !q_dev || !out_dev) return VEDT_EINVAL;
    if (!n->fused_valid) {   // parameters changed on the device (training): fetch the biases once
        for (int l = 0; l < kLayers - 1; ++l)
            MCHECK(cudaMemcpyAsync(n->fused.bias[l], n->p + n->offB[l], sizeof(float) * kHidden, cudaMemcpyDeviceToHost,
                                   n->stream));
        MCHECK(cudaMemcpyAsync(n->fused.bias_out, n->p + n->offB[kLayers - 1], sizeof(float) * kOutPad,
                               cudaMemcpyDeviceToHost, n->stream));
        MCHECK(cudaStreamSynchronize(n->stream));
        n->fused.wimg = n->wimg;
        n->fused_valid = true;
    }
    MCHECK(launch_fused(n, q_dev, B, n->fused, out_dev));
    return VEDT_OK;
}

// Layer-by-layer forward (the training path's), kept for comparison.
vedt_status vedt_mlp_forward_layers(vedt_mlp *n, const float *q_dev, int B, float *out_dev) {
    if (!check_rows(n, B) || !q_dev || !out_dev) return VEDT_EINVAL;
    const int rows = (B + 127) / 128 * 128;
    vedt_status st = features(n, q_dev, B, rows);
    if (st == VEDT_OK) st = forward_rows(n, rows);
    if (st != VEDT_OK) return st;
    k_copy_out<<<(B * kOut + 255) / 256, 256, 0, n->stream>>>(n->out, B, out_dev);
    MCHECK(cudaGetLastError());
    return VEDT_OK;
}

vedt_status vedt_mlp_grads(vedt_mlp *n, const float *q_dev, const float *y_dev, const float *mask_dev, int B,
                           float *grads_host, int64_t count, float *loss_host) {
    if (!check_rows(n, B) || !q_dev || !y_dev || !grads_host) return VEDT_EINVAL;
    const int rows = (B + 127) / 128 * 128;
    vedt_status st = features(n, q_dev, B, rows);
    if (st == VEDT_OK) st = forward_rows(n, rows);
    if (st == VEDT_OK) st = backward(n, y_dev, mask_dev, B, rows);
    if (st != VEDT_OK) return st;
    st = unpad(n, n->g, grads_host, count);
    if (st != VEDT_OK) return st;
    if (loss_host) {
        float sums[2];
        MCHECK(cudaMemcpy(sums, n->sums, sizeof(sums), cudaMemcpyDeviceToHost));
        *loss_host = sums[0] / std::max(sums[1], 1.0f);
    }
    return VEDT_OK;
}

vedt_status vedt_mlp_train_step(vedt_mlp *n, const float *q_dev, const float *y_dev, const float *mask_dev, int B,
                                float lr, float wd, float *loss_sums_dev) {
    if (!check_rows(n, B) || !q_dev || !y_dev || !(lr >= 0.f) || !(wd >= 0.f)) return VEDT_EINVAL;
    const int rows = (B + 127) / 128 * 128;
    vedt_status st = features(n, q_dev, B, rows);
    if (st == VEDT_OK) st = forward_rows(n, rows);
    if (st == VEDT_OK) st = backward(n, y_dev, mask_dev, B, rows);
    if (st != VEDT_OK) return st;
    n->step += 1;
    n->fused_valid = false;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, static_cast<float>(n->step));
    const float c2 = 1.f - std::pow(b2, static_cast<float>(n->step));
    k_adamw<<<static_cast<unsigned>((n->np + 255) / 256), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->np, lr, wd,
                                                                               b1, b2, 1e-8f, c1, c2);
    MCHECK(cudaGetLastError());
    if (loss_sums_dev) MCHECK(cudaMemcpyAsync(loss_sums_dev, n->sums, 2 * sizeof(float), cudaMemcpyDeviceToDevice,
                                              n->stream));
    return refresh_bf16(n);
}

vedt_status vedt_mlp_check(vedt_mlp *n) {
    if (!n) return VEDT_EINVAL;
    MCHECK(cudaStreamSynchronize(n->stream));
    int32_t e = 0;
    MCHECK(cudaMemcpy(&e, n->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) {
        MCHECK(cudaMemset(n->err, 0, sizeof(int32_t)));
        return VEDT_ETIMEOUT;
    }
    return VEDT_OK;
}

}  // extern "C"
