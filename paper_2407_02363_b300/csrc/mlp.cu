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

#include <cmath>
#include <cstring>
#include <new>
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
// One CTA computes all five layers for 128 rows.  The activation tile (128 x 256 bf16)
// stays in shared memory in the canonical K-major layout (SBO 4096 B); weights stream in
// K chunks of 32 columns (all N rows) through two cp.async buffers; chunk g of the whole
// forward uses buffer g % 2, its MMAs commit to that buffer's mbarrier, and the buffer is
// refilled only after that commit completed (parity (g / 2) & 1).
struct FusedArgs {
    const bf16 *w[kLayers];     // [N_l][K_l] row-major bf16
    const float *b[kLayers];    // [N_l] fp32
};

constexpr int kFKC = 32;                    // weight K chunk
constexpr int kActBytes = 128 * kHidden * 2;
constexpr int kFeatBytes = 128 * kInPad * 2;
constexpr int kWBufBytes = kHidden * kFKC * 2;
constexpr int kFusedSmem = kActBytes + kFeatBytes + 2 * kWBufBytes;
constexpr int kChunks = 1 + (kLayers - 1) * (kHidden / kFKC);   // 33

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// layer and K-chunk of global chunk index g
__device__ __forceinline__ void chunk_of(int g, int &l, int &kc) {
    if (g == 0) {
        l = 0;
        kc = 0;
    } else {
        l = 1 + (g - 1) / (kHidden / kFKC);
        kc = (g - 1) % (kHidden / kFKC);
    }
}

// stages weight chunk g (rows 0..N_l-1, K columns of the chunk) into buf, canonical layout
__device__ __forceinline__ void stage_w(const FusedArgs &a, int g, uint8_t *buf) {
    int l, kc;
    chunk_of(g, l, kc);
    const int N = layer_n(l), K = layer_k(l);
    const int kw = (l == 0) ? kInPad : kFKC;    // chunk width in elements
    const int kv = kw / 8;
    const int V = N * kv;
    const bf16 *W = a.w[l];
    for (int v = threadIdx.x; v < V; v += kThreads) {
        const int rr = v & 7, gg = v >> 3;
        const int r = (gg / kv) * 8 + rr, k8 = gg % kv;
        cp_async16(buf + 16 * v, W + static_cast<int64_t>(r) * K + kc * kFKC + 8 * k8);
    }
}

__global__ void __launch_bounds__(kThreads) k_mlp_fused(const float *__restrict__ q, int B, FusedArgs a,
                                                        float *__restrict__ out, int32_t *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    uint8_t *act = smem;
    uint8_t *feat = smem + kActBytes;
    uint8_t *wbuf[2] = {feat + kFeatBytes, feat + kFeatBytes + kWBufBytes};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = blockIdx.x * 128 + tid;     // feature row of this thread
    if (warp == 0) tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    // features [sin q, cos q, 0, 0] of row `tid` in the canonical layout (kv = 2)
    {
        alignas(16) bf16 f[kInPad];
        for (int j = 0; j < kInPad; ++j) {
            float val = 0.f;
            if (row < B && j < kIn) val = j < 7 ? sinf(q[row * 7 + j]) : cosf(q[row * 7 + j - 7]);
            f[j] = __float2bfloat16_rn(val);
        }
        const int base = (tid >> 3) * 2 * 128 + (tid & 7) * 16;
        *reinterpret_cast<uint4 *>(feat + base) = *reinterpret_cast<const uint4 *>(f);
        *reinterpret_cast<uint4 *>(feat + base + 128) = *reinterpret_cast<const uint4 *>(f + 8);
    }
    stage_w(a, 0, wbuf[0]);
    cp_async_commit();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    bool ok = true;
    for (int g = 0; g < kChunks && ok; ++g) {
        int l, kc;
        chunk_of(g, l, kc);
        const int N = layer_n(l);
        // refill the other buffer with chunk g+1 once chunk g-1's MMAs released it
        if (g + 1 < kChunks) {
            if (g >= 1) ok = mbar_wait_bounded(&mbar[(g + 1) & 1], ((g - 1) >> 1) & 1, err);
            stage_w(a, g + 1, wbuf[(g + 1) & 1]);
        }
        cp_async_commit();
        cp_async_wait_1();                       // chunk g has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            if (l == 0) {
                const uint64_t da = smem_desc(smem_u32(feat), 128, 256);
                const uint64_t db = smem_desc(smem_u32(wbuf[0]), 128, 256);
                mma_bf16(taddr, da, db, idesc_bf16(128, kHidden), 0u);
            } else {
                const uint32_t idesc = idesc_bf16(128, N);
                for (int s = 0; s < kFKC / 16; ++s) {
                    const int k16 = kc * (kFKC / 16) + s;
                    const uint64_t da = smem_desc(smem_u32(act + k16 * 256), 128, (kHidden / 8) * 128);
                    const uint64_t db = smem_desc(smem_u32(wbuf[g & 1] + s * 256), 128, (kFKC / 8) * 128);
                    mma_bf16(taddr, da, db, idesc, (kc > 0 || s > 0) ? 1u : 0u);
                }
            }
            mma_commit(&mbar[g & 1]);
        }
        const bool last = (l == 0) || (kc == kHidden / kFKC - 1);
        if (!last || !ok) continue;
        // layer done: wait for its MMAs, then epilogue from TMEM
        ok = mbar_wait_bounded(&mbar[g & 1], (g >> 1) & 1, err);
        if (!ok) break;
        tc_fence_after();
        const int r = blockIdx.x * 128 + warp * 32 + lane;
        const int rl = warp * 32 + lane;       // row within the tile = TMEM lane
        if (l < kLayers - 1) {
            for (int c0 = 0; c0 < kHidden; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
                alignas(16) bf16 h[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(fmaxf(v[i] + a.b[l][c0 + i], 0.0f));
                const int base = ((rl >> 3) * (kHidden / 8) + (c0 >> 3)) * 128 + (rl & 7) * 16;
                *reinterpret_cast<uint4 *>(act + base) = *reinterpret_cast<const uint4 *>(h);
                *reinterpret_cast<uint4 *>(act + base + 128) = *reinterpret_cast<const uint4 *>(h + 8);
            }
        } else {
            for (int c0 = 0; c0 < kOutPad; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
                if (r < B) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < kOut) out[static_cast<int64_t>(r) * kOut + c0 + i] = v[i] + a.b[l][c0 + i];
                }
            }
        }
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        tc_fence_after();
    }
    cp_async_wait_0();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 256);
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
    cudaError_t e = cudaFuncSetAttribute(k_gemm<N, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
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

vedt_status vedt_mlp_set_params(vedt_mlp *n, const float *params, int64_t count) {
    if (!n || !params || count != vedt_mlp_num_params()) return VEDT_EINVAL;
    std::vector<float> pad(static_cast<size_t>(n->np), 0.f);
    int64_t r = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int Nv = layer_n_valid(l), Kv = layer_k_valid(l), K = layer_k(l);
        for (int i = 0; i < Nv; ++i)
            for (int k = 0; k < Kv; ++k) pad[n->offW[l] + static_cast<int64_t>(i) * K + k] = params[r++];
        for (int i = 0; i < Nv; ++i) pad[n->offB[l] + i] = params[r++];
    }
    MCHECK(cudaMemcpyAsync(n->p, pad.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice, n->stream));
    MCHECK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->np, n->stream));
    MCHECK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->np, n->stream));
    n->step = 0;
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

vedt_status vedt_mlp_forward(vedt_mlp *n, const float *q_dev, int B, float *out_dev) {
    if (!check_rows(n, B) || !q_dev || !out_dev) return VEDT_EINVAL;
    FusedArgs a{};
    for (int l = 0; l < kLayers; ++l) {
        a.w[l] = n->wb[l];
        a.b[l] = n->p + n->offB[l];
    }
    MCHECK(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem));
    k_mlp_fused<<<(B + 127) / 128, kThreads, kFusedSmem, n->stream>>>(q_dev, B, a, out_dev, n->err);
    MCHECK(cudaGetLastError());
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
