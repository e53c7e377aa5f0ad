// Learned Newton seed: the small MLP of bspl_mlp.h on the tensor cores.
//
// Inference (k_mlp_fused): one persistent block per SM of four warpgroups.
// The BF16 weights of the three 128-wide layers stay in shared memory; each
// warpgroup runs its own tiles of 128 rows: inputs -> shared memory (BF16) ->
// tcgen05.mma into its 128 tensor-memory columns -> tcgen05.ld, bias, GELU,
// BF16 -> shared memory -> next layer; the last layer's epilogue also takes
// the dot product with w4 and the sigmoid.  One thread per warpgroup issues
// the MMAs; completion comes back through an mbarrier.
//
// Training: the same arithmetic split into a generic tcgen05 GEMM
// (C = A B^T, BF16 operands staged by the threads, FP32 accumulators in
// tensor memory, optional split-K with FP32 atomics) plus element-wise
// kernels for bias, GELU and its derivative, the output layer, transposes
// and Adam.
#include <math.h>

#include "../../include/bspl_mlp.h"
#include "query_common.cuh"
#include "tc05.cuh"

namespace bspl {
namespace {

constexpr int kH = BSPL_MLP_HIDDEN;
constexpr int kBfW1 = 0, kBfW2 = 2048, kBfW3 = 2048 + 16384, kBfW2T = 2048 + 2 * 16384, kBfW3T = 2048 + 3 * 16384,
              kBfW4 = 2048 + 4 * 16384;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s bound on every mbarrier wait

// set when a tensor-core wait gave up (read and cleared by bspl_mlp_check)
__device__ int g_tc_timeout;

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
}

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// ------------------------------------------------------------ BF16 weights
__global__ void k_sync(const float* __restrict__ p, uint16_t* __restrict__ w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BSPL_MLP_NBF16) return;
    float v;
    if (i < kBfW2) v = p[BSPL_MLP_OFF_W1 + i];
    else if (i < kBfW3) v = p[BSPL_MLP_OFF_W2 + (i - kBfW2)];
    else if (i < kBfW2T) v = p[BSPL_MLP_OFF_W3 + (i - kBfW3)];
    else if (i < kBfW3T) {
        int j = i - kBfW2T, r = j / kH, c = j % kH;  // W2^T[r][c] = W2[c][r]
        v = p[BSPL_MLP_OFF_W2 + c * kH + r];
    } else if (i < kBfW4) {
        int j = i - kBfW3T, r = j / kH, c = j % kH;
        v = p[BSPL_MLP_OFF_W3 + c * kH + r];
    } else v = p[BSPL_MLP_OFF_W4 + (i - kBfW4)];
    w[i] = f2bf(v);
}

// ------------------------------------------------------------ pair features
// Inputs of a (query, segment) pair in the frame of the segment's control-
// point box, all in FP32: control points relative to P0 come from the power
// coefficients (P1 - P0 = a1/3, P2 - P0 = (2 a1 + a2)/3, P3 - P0 =
// a1 + a2 + a3), so short segments keep their relative accuracy; q - P0
// from the high and low FP32 parts of both (qr: q hi[3], q lo[3]).  The
// query keeps its coordinate along the chord P0 -> P3 (which fixes the
// minimiser of a far query); its part across the chord is shortened to
// length min(1, |part|).
__device__ __forceinline__ void pair_features(const float* __restrict__ r32, const float* qr, float f[16])
{
    float d[4][3], cc[3];
    float ext = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a1 = r32[9 + c], a2 = r32[12 + c], a3 = r32[15 + c];
        d[0][c] = 0.f;
        d[1][c] = a1 / 3.f;
        d[2][c] = (2.f * a1 + a2) / 3.f;
        d[3][c] = a1 + a2 + a3;
        const float lo = fminf(fminf(d[0][c], d[1][c]), fminf(d[2][c], d[3][c]));
        const float hi = fmaxf(fmaxf(d[0][c], d[1][c]), fmaxf(d[2][c], d[3][c]));
        cc[c] = 0.5f * (lo + hi);
        ext = fmaxf(ext, hi - lo);
    }
    const float s = ext > 0.f ? 1.f / ext : 1.f;
    float v[3], dn[3];
    const float ln = sqrtf(d[3][0] * d[3][0] + d[3][1] * d[3][1] + d[3][2] * d[3][2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int i = 0; i < 4; ++i) f[3 * i + c] = (d[i][c] - cc[c]) * s;
        const float qm = (qr[c] - r32[6 + c]) + (qr[3 + c] - r32[18 + c]);  // q - P0
        v[c] = (qm - cc[c]) * s;
        dn[c] = ln > 0.f ? d[3][c] / ln : (c == 0 ? 1.f : 0.f);
    }
    const float a = v[0] * dn[0] + v[1] * dn[1] + v[2] * dn[2];
    const float w0 = v[0] - a * dn[0], w1 = v[1] - a * dn[1], w2 = v[2] - a * dn[2];
    const float k = 1.f / fmaxf(1.f, sqrtf(w0 * w0 + w1 * w1 + w2 * w2));
    f[12] = a * dn[0] + w0 * k;
    f[13] = a * dn[1] + w1 * k;
    f[14] = a * dn[2] + w2 * k;
    f[15] = 0.f;
}

struct SrcX {
    const float* X;
    int64_t n;
    __device__ int64_t count() const { return n; }
    __device__ void features(int64_t i, float f[16]) const
    {
        const float4* p = reinterpret_cast<const float4*>(X + 16 * i);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 v = p[k];
            f[4 * k] = v.x;
            f[4 * k + 1] = v.y;
            f[4 * k + 2] = v.z;
            f[4 * k + 3] = v.w;
        }
    }
};

}  // namespace

// the learned path's seed pairs [0, min(cap, *n_dev)) of (query, segment)
struct SrcPairs {
    const int32_t* pq;  // sorted query position
    const int32_t* ps;
    const float* qrec;  // per sorted query: q hi[3], q lo[3], ...
    const float* rec32;
    int64_t cap;
    const unsigned long long* n_dev;
    __device__ int64_t count() const { return min(cap, (int64_t)*n_dev); }
    __device__ void features(int64_t i, float f[16]) const
    {
        pair_features(rec32 + (int64_t)BSPL_CREC32 * ps[i], qrec + 8 * (int64_t)pq[i], f);
    }
};

namespace {

// ------------------------------------------------------- fused inference
constexpr int kFusedWG = 4;  // warpgroups per block
constexpr int kSmW1 = 0, kSmW2 = 4096, kSmW3 = kSmW2 + 32768, kSmBias = kSmW3 + 32768;  // bias: 4 x 128 + 1 floats
constexpr int kSmF = kSmBias + 2560, kSmX = kSmF + kFusedWG * 4096, kSmBar = kSmX + kFusedWG * 32768;
constexpr int kSmFusedBytes = kSmBar + 64;

// a [rows][K] bf16 row-major matrix -> core-matrix layout (see tc05.cuh)
__device__ __forceinline__ void stage_weights(uint8_t* dst, const uint16_t* __restrict__ src, int rows, int K,
                                              int tid, int nthreads)
{
    const int kgs = K / 8;
    for (int c = tid; c < rows * kgs; c += nthreads) {
        const int r = c / kgs, kg = c % kgs;
        const uint4 v = *reinterpret_cast<const uint4*>(src + (int64_t)r * K + kg * 8);
        *reinterpret_cast<uint4*>(dst + (r >> 3) * K * 16 + kg * 128 + (r & 7) * 16) = v;
    }
}

// bias + GELU of the 128 accumulators of this thread's row -> BF16 row of X
__device__ __forceinline__ void epi_hidden(uint32_t tl, const float* b, uint8_t* X, int r)
{
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
        float v[32];
        tc::tmem_ld32(tl + cb * 32, v);
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            pk[j] = tc::pack_bf16(tc::gelu(v[2 * j] + b[cb * 32 + 2 * j]), tc::gelu(v[2 * j + 1] + b[cb * 32 + 2 * j + 1]));
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(X + (r >> 3) * kH * 16 + (cb * 4 + q) * 128 + (r & 7) * 16) =
                make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}

template <class Src>
__global__ void __launch_bounds__(kFusedWG * 128, 1)
    k_mlp_fused(Src src, const uint16_t* __restrict__ wb, const float* __restrict__ params, float* __restrict__ out)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kSmBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSmBar + 8 * kFusedWG);
    volatile int* okf = reinterpret_cast<volatile int*>(sm + kSmBar + 8 * kFusedWG + 8);
    float* bias = reinterpret_cast<float*>(sm + kSmBias);
    const int tid = threadIdx.x, g = tid >> 7, r = tid & 127, warp = tid >> 5;

    if (warp == 0) {
        tc::tmem_alloc(tslot, 512);
        tc::tmem_relinquish();
    }
    if (tid < kFusedWG) {
        tc::mbar_init(&mbar[tid], 1);
        tc::fence_mbar_init();
        okf[tid] = 1;
    }
    stage_weights(sm + kSmW1, wb + kBfW1, kH, 16, tid, blockDim.x);
    stage_weights(sm + kSmW2, wb + kBfW2, kH, kH, tid, blockDim.x);
    stage_weights(sm + kSmW3, wb + kBfW3, kH, kH, tid, blockDim.x);
    for (int i = tid; i < 3 * kH; i += blockDim.x) {
        const int l = i / kH, c = i % kH;
        const int off = l == 0 ? BSPL_MLP_OFF_B1 : (l == 1 ? BSPL_MLP_OFF_B2 : BSPL_MLP_OFF_B3);
        bias[i] = params[off + c];
    }
    for (int i = tid; i < kH; i += blockDim.x) bias[3 * kH + i] = bf2f(wb[kBfW4 + i]);
    if (tid == 0) bias[4 * kH] = params[BSPL_MLP_OFF_B4];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t tacc = *tslot + (uint32_t)(g * 128);
    const uint32_t tl = tacc + ((uint32_t)((warp & 3) * 32) << 16);
    uint8_t* F = sm + kSmF + g * 4096;
    uint8_t* X = sm + kSmX + g * 32768;
    const uint32_t aF = tc::smem_u32(F), aX = tc::smem_u32(X);
    const uint32_t aW1 = tc::smem_u32(sm + kSmW1), aW2 = tc::smem_u32(sm + kSmW2), aW3 = tc::smem_u32(sm + kSmW3);
    constexpr uint32_t idesc = tc::idesc_bf16(128, kH);
    const float* w4 = bias + 3 * kH;
    const float b4 = bias[4 * kH];
    const int bar_id = 1 + g;
    uint32_t phase = 0;

    const int64_t n = src.count();
    const int64_t ntiles = (n + 127) / 128;
    // one MMA group, completion awaited by the issuing thread, result shared
    auto run_layer = [&](int layer) -> bool {
        if (r == 0) {
            tc::fence_after_sync();
            if (layer == 0) {
                tc::mma_bf16(tacc, tc::sdesc(aF, 128, 256), tc::sdesc(aW1, 128, 256), idesc, 0);
            } else {
                const uint32_t aW = layer == 1 ? aW2 : aW3;
#pragma unroll
                for (int ks = 0; ks < kH / 16; ++ks)
                    tc::mma_bf16(tacc, tc::sdesc(aX + ks * 256, 128, kH * 16), tc::sdesc(aW + ks * 256, 128, kH * 16),
                                 idesc, ks > 0);
            }
            tc::mma_commit(&mbar[g]);
            if (!tc::mbar_wait(&mbar[g], phase, kWaitNs)) {
                okf[g] = 0;
                atomicExch(&g_tc_timeout, 1);
            }
        }
        phase ^= 1;
        named_sync(bar_id, 128);
        tc::fence_after_sync();
        return okf[g] != 0;
    };

    for (int64_t tile = (int64_t)blockIdx.x * kFusedWG + g; tile < ntiles; tile += (int64_t)gridDim.x * kFusedWG) {
        const int64_t i = tile * 128 + r;
        float f[16];
        if (i < n) src.features(i, f);
        else {
#pragma unroll
            for (int k = 0; k < 16; ++k) f[k] = 0.f;
        }
        *reinterpret_cast<uint4*>(F + (r >> 3) * 256 + (r & 7) * 16) =
            make_uint4(tc::pack_bf16(f[0], f[1]), tc::pack_bf16(f[2], f[3]), tc::pack_bf16(f[4], f[5]),
                       tc::pack_bf16(f[6], f[7]));
        *reinterpret_cast<uint4*>(F + (r >> 3) * 256 + 128 + (r & 7) * 16) =
            make_uint4(tc::pack_bf16(f[8], f[9]), tc::pack_bf16(f[10], f[11]), tc::pack_bf16(f[12], f[13]),
                       tc::pack_bf16(f[14], f[15]));
        tc::fence_async_smem();
        tc::fence_before_sync();
        named_sync(bar_id, 128);
        if (!run_layer(0)) break;
        epi_hidden(tl, bias, X, r);
        tc::fence_async_smem();
        tc::fence_before_sync();
        named_sync(bar_id, 128);
        if (!run_layer(1)) break;
        epi_hidden(tl, bias + kH, X, r);
        tc::fence_async_smem();
        tc::fence_before_sync();
        named_sync(bar_id, 128);
        if (!run_layer(2)) break;
        float z = b4;
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
            float v[32];
            tc::tmem_ld32(tl + cb * 32, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = cb * 32 + j;
                z = fmaf(bf2f(f2bf(tc::gelu(v[j] + bias[2 * kH + c]))), w4[c], z);
            }
        }
        if (i < n) out[i] = 1.f / (1.f + __expf(-z));
        tc::fence_before_sync();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(*tslot, 512);
    }
}

// ------------------------------------------------------------ generic GEMM
// C[M][N] (+)= A[M][K] B[N][K]^T, A and B BF16 row-major (lda, ldb multiples
// of 8 elements, 16-byte aligned), K a multiple of 16; block (mt, nt, ks)
// covers rows mt*128.., columns nt*128.. and K range [ks*kps, (ks+1)*kps).
constexpr int kGemmSmem = 65536;  // requested so that at most 3 blocks share an SM's tensor memory

__global__ void __launch_bounds__(128) k_gemm_nt(const uint16_t* __restrict__ A, int64_t lda,
                                                 const uint16_t* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                                 int64_t ldc, int M, int N, int K, int kps, int atomic)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* As = sm;
    uint8_t* Bs = sm + 16384;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 32768);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 32768 + 8);
    volatile int* okf = reinterpret_cast<volatile int*>(sm + 32768 + 16);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
    const int kb = blockIdx.z * kps, ke = min(K, kb + kps);
    if (warp == 0) {
        tc::tmem_alloc(tslot, 128);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
        *okf = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tacc = *tslot;
    const uint32_t aA = tc::smem_u32(As), aB = tc::smem_u32(Bs);
    constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
    uint32_t phase = 0;
    bool any = false, ok = true;
    for (int k0 = kb; k0 < ke && ok; k0 += 64) {
        const int kc = min(64, ke - k0);
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (kg * 8 < kc) {
                if (m0 + t < M) va = *reinterpret_cast<const uint4*>(A + (int64_t)(m0 + t) * lda + k0 + kg * 8);
                if (n0 + t < N) vb = *reinterpret_cast<const uint4*>(B + (int64_t)(n0 + t) * ldb + k0 + kg * 8);
            }
            const int off = (t >> 3) * 1024 + kg * 128 + (t & 7) * 16;
            *reinterpret_cast<uint4*>(As + off) = va;
            *reinterpret_cast<uint4*>(Bs + off) = vb;
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            for (int ks = 0; ks < kc / 16; ++ks)
                tc::mma_bf16(tacc, tc::sdesc(aA + ks * 256, 128, 1024), tc::sdesc(aB + ks * 256, 128, 1024), idesc,
                             (any || ks > 0) ? 1u : 0u);
            tc::mma_commit(mbar);
            if (!tc::mbar_wait(mbar, phase, kWaitNs)) {
                *okf = 0;
                atomicExch(&g_tc_timeout, 1);
            }
        }
        phase ^= 1;
        any = true;
        __syncthreads();
        tc::fence_after_sync();
        ok = *okf != 0;
    }
    if (ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
            float v[32];
            if (any) tc::tmem_ld32(tacc + ((uint32_t)(warp * 32) << 16) + cb * 32, v);
            else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
            }
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + cb * 32 + j;
                    if (col < N) {
                        if (atomic) atomicAdd(C + (int64_t)row * ldc + col, v[j]);
                        else C[(int64_t)row * ldc + col] = v[j];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tacc, 128);
    }
}

cudaError_t gemm_nt(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int M,
                    int N, int K, int splits, bool atomic, cudaStream_t s)
{
    int kps = (K + splits - 1) / splits;
    kps = (kps + 63) / 64 * 64;
    splits = (K + kps - 1) / kps;
    dim3 grid((M + 127) / 128, (N + 127) / 128, splits);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    k_gemm_nt<<<grid, 128, kGemmSmem, s>>>(A, lda, B, ldb, C, ldc, M, N, K, kps, atomic ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------ training kernels
// rows of the batch: row i < nvalid takes source row src_row(i), others 0
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ y, int64_t n, int64_t start,
                         uint64_t a, uint64_t b, int nvalid, int Bp, uint16_t* __restrict__ Xb,
                         uint16_t* __restrict__ XT, float* __restrict__ yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp) return;
    float f[16];
    float yy = 0.f;
    if (i < nvalid) {
        const uint64_t x = (uint64_t)(start + i) % (uint64_t)n;
        const uint64_t j = (a * x % (uint64_t)n + b) % (uint64_t)n;
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = X[16 * (int64_t)j + k];
        yy = y[j];
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint16_t h = f2bf(f[k]);
        Xb[16 * i + k] = h;
        XT[(int64_t)k * Bp + i] = h;
    }
    yb[i] = yy;
}

// Z += b (kept as the pre-activation), H = bf16(GELU(Z)), HT = H^T; 32x32 tiles
__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ b, uint16_t* __restrict__ Hb,
                           uint16_t* __restrict__ HT, int Bp)
{
    __shared__ uint16_t tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += blockDim.y) {
        const int64_t idx = (int64_t)(r0 + k) * kH + c0 + tx;
        const float z = Z[idx] + b[c0 + tx];
        Z[idx] = z;
        const uint16_t h = f2bf(tc::gelu(z));
        Hb[idx] = h;
        tile[k][tx] = h;
    }
    if (!HT) return;
    __syncthreads();
    for (int k = ty; k < 32; k += blockDim.y) HT[(int64_t)(c0 + k) * Bp + r0 + tx] = tile[tx][k];
}

// output layer: z4 = H3 . w4 + b4, t = sigmoid, loss, dz4 (one warp per row)
__global__ void k_head(const uint16_t* __restrict__ H3, const uint16_t* __restrict__ wb,
                       const float* __restrict__ params, const float* __restrict__ yb, int nvalid, int Bp,
                       float loss_scale, float* __restrict__ dz4, float* __restrict__ loss)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= Bp) return;
    float z = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = lane + 32 * k;
        z += bf2f(H3[(int64_t)row * kH + c]) * bf2f(wb[kBfW4 + c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) {
        z += params[BSPL_MLP_OFF_B4];
        const float t = 1.f / (1.f + __expf(-z));
        float d = 0.f;
        if (row < nvalid) {
            const float rr = t - yb[row];
            d = 2.f / (float)nvalid * rr * t * (1.f - t);
            atomicAdd(loss, rr * rr * loss_scale);
        }
        dz4[row] = d;
    }
}

// dZ = dH (.) GELU'(Z) with dH = dz4 w4^T (head) or the GEMM output; writes
// BF16 dZ and its transpose; column sums of dZ -> bias gradient; for the
// head also the w4 and b4 gradients
template <bool HEAD>
__global__ void k_act_back(const float* __restrict__ dH, const float* __restrict__ dz4,
                           const uint16_t* __restrict__ H3, const uint16_t* __restrict__ wb,
                           const float* __restrict__ Z, uint16_t* __restrict__ dZb, uint16_t* __restrict__ dZT,
                           float* __restrict__ gbias, float* __restrict__ gw4, float* __restrict__ gb4, int Bp)
{
    __shared__ uint16_t tile[32][33];
    __shared__ float csum[8][32], cw4[8][32], cb4[8];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float sb = 0.f, sw = 0.f, s4 = 0.f;
    for (int k = ty; k < 32; k += blockDim.y) {
        const int row = r0 + k, col = c0 + tx;
        const int64_t idx = (int64_t)row * kH + col;
        float g;
        if (HEAD) {
            const float d4 = dz4[row];
            g = d4 * bf2f(wb[kBfW4 + col]);
            sw += d4 * bf2f(H3[idx]);
            if (tx == 0) s4 += d4;
        } else g = dH[idx];
        const float dz = g * tc::gelu_grad(Z[idx]);
        sb += dz;
        const uint16_t h = f2bf(dz);
        dZb[idx] = h;
        tile[k][tx] = h;
    }
    csum[ty][tx] = sb;
    cw4[ty][tx] = sw;
    if (tx == 0) cb4[ty] = s4;
    __syncthreads();
    for (int k = ty; k < 32; k += blockDim.y) dZT[(int64_t)(c0 + k) * Bp + r0 + tx] = tile[tx][k];
    if (ty == 0) {
        float a = 0.f, w = 0.f;
        for (int k = 0; k < (int)blockDim.y; ++k) {
            a += csum[k][tx];
            w += cw4[k][tx];
        }
        atomicAdd(gbias + c0 + tx, a);
        if (HEAD) atomicAdd(gw4 + c0 + tx, w);
        if (HEAD && tx == 0 && blockIdx.y == 0) {
            float s = 0.f;
            for (int k = 0; k < (int)blockDim.y; ++k) s += cb4[k];
            atomicAdd(gb4, s);
        }
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_features(const bspl_segments S, int64_t n, const int32_t* __restrict__ pq,
                           const int32_t* __restrict__ ps, const double* __restrict__ q_xyz, float* __restrict__ X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[16];
    const int64_t s = ps[i];
    if (s < 0 || s >= S.capacity || pq[i] < 0) {
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = __int_as_float(0x7fc00000);
    } else {
        const double* q = q_xyz + 3 * (int64_t)pq[i];
        float qr[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            qr[k] = (float)q[k];
            qr[3 + k] = (float)(q[k] - (double)qr[k]);
        }
        pair_features(S.rec32 + (int64_t)BSPL_CREC32 * s, qr, f);
    }
    float4* o = reinterpret_cast<float4*>(X + 16 * i);
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

__global__ void k_labels(const bspl_segments S, int64_t n, const int32_t* __restrict__ pq,
                         const int32_t* __restrict__ ps, const double* __restrict__ q_xyz, float* __restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = ps[i];
    if (s < 0 || s >= S.capacity || pq[i] < 0) {
        y[i] = __int_as_float(0x7fc00000);
        return;
    }
    const double* a = S.rec64 + (int64_t)BSPL_CREC64 * s + 6;
    const double* q = q_xyz + 3 * (int64_t)pq[i];
    double c[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) c[k] = a[k];
    c[0] -= q[0];
    c[1] -= q[1];
    c[2] -= q[2];
    y[i] = (float)isolate_min<double>(c, 0.0, 0.0, 0.0, 1e-15, 200);
}

// workspace of one training batch of Bp rows (multiple of 128)
struct TrainWs {
    uint16_t *Xb, *XT, *H1, *H2, *H3, *H1T, *H2T, *dZb, *dZT;
    float *yb, *Z1, *Z2, *Z3, *dz4, *dH, *grad, *loss;
};

TrainWs carve_train(Carver& cv, int Bp)
{
    TrainWs w{};
    w.Xb = cv.take<uint16_t>((size_t)Bp * 16);
    w.XT = cv.take<uint16_t>((size_t)Bp * 16);
    w.yb = cv.take<float>((size_t)Bp);
    w.Z1 = cv.take<float>((size_t)Bp * kH);
    w.Z2 = cv.take<float>((size_t)Bp * kH);
    w.Z3 = cv.take<float>((size_t)Bp * kH);
    w.H1 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H2 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H3 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H1T = cv.take<uint16_t>((size_t)Bp * kH);
    w.H2T = cv.take<uint16_t>((size_t)Bp * kH);
    w.dz4 = cv.take<float>((size_t)Bp);
    w.dH = cv.take<float>((size_t)Bp * kH);
    w.dZb = cv.take<uint16_t>((size_t)Bp * kH);
    w.dZT = cv.take<uint16_t>((size_t)Bp * kH);
    w.grad = cv.take<float>(BSPL_MLP_NPARAM);
    w.loss = cv.take<float>(4);
    return w;
}

int padded(int64_t batch) { return (int)((batch + 127) / 128 * 128); }

// forward + backward of one padded batch already gathered into w (Xb, XT,
// yb); grad overwritten, loss_scale * sum of squared residuals added to *loss
cudaError_t batch_grad(const bspl_mlp* m, const TrainWs& w, float* grad, int nvalid, int Bp, float loss_scale,
                       float* loss, cudaStream_t s)
{
    const uint16_t* wb = m->wbf16;
    const float* p = m->params;
    float* g = grad;
    cudaError_t e = cudaMemsetAsync(g, 0, sizeof(float) * BSPL_MLP_NPARAM, s);
    if (e != cudaSuccess) return e;
    const dim3 tb(32, 8), tg(Bp / 32, kH / 32);
    const int splits = std::max(1, Bp / 512);
    // forward: Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l)
    if ((e = gemm_nt(w.Xb, 16, wb + kBfW1, 16, w.Z1, kH, Bp, kH, 16, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z1, p + BSPL_MLP_OFF_B1, w.H1, w.H1T, Bp);
    if ((e = gemm_nt(w.H1, kH, wb + kBfW2, kH, w.Z2, kH, Bp, kH, kH, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z2, p + BSPL_MLP_OFF_B2, w.H2, w.H2T, Bp);
    if ((e = gemm_nt(w.H2, kH, wb + kBfW3, kH, w.Z3, kH, Bp, kH, kH, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z3, p + BSPL_MLP_OFF_B3, w.H3, nullptr, Bp);
    k_head<<<Bp / 8, 256, 0, s>>>(w.H3, wb, p, w.yb, nvalid, Bp, loss_scale, w.dz4, loss);
    // layer 3: dZ3 = (dz4 w4^T) (.) GELU'(Z3); dW3 = dZ3^T H2; dH2 = dZ3 W3
    k_act_back<true><<<tg, tb, 0, s>>>(nullptr, w.dz4, w.H3, wb, w.Z3, w.dZb, w.dZT, g + BSPL_MLP_OFF_B3,
                                       g + BSPL_MLP_OFF_W4, g + BSPL_MLP_OFF_B4, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.H2T, Bp, g + BSPL_MLP_OFF_W3, kH, kH, kH, Bp, splits, true, s))) return e;
    if ((e = gemm_nt(w.dZb, kH, wb + kBfW3T, kH, w.dH, kH, Bp, kH, kH, 1, false, s))) return e;
    // layer 2
    k_act_back<false><<<tg, tb, 0, s>>>(w.dH, nullptr, nullptr, wb, w.Z2, w.dZb, w.dZT, g + BSPL_MLP_OFF_B2,
                                        nullptr, nullptr, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.H1T, Bp, g + BSPL_MLP_OFF_W2, kH, kH, kH, Bp, splits, true, s))) return e;
    if ((e = gemm_nt(w.dZb, kH, wb + kBfW2T, kH, w.dH, kH, Bp, kH, kH, 1, false, s))) return e;
    // layer 1: dW1 = dZ1^T X (N = 16 columns)
    k_act_back<false><<<tg, tb, 0, s>>>(w.dH, nullptr, nullptr, wb, w.Z1, w.dZb, w.dZT, g + BSPL_MLP_OFF_B1,
                                        nullptr, nullptr, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.XT, Bp, g + BSPL_MLP_OFF_W1, 16, kH, 16, Bp, splits, true, s))) return e;
    return cudaGetLastError();
}

cudaError_t launch_adam(const bspl_mlp* m, const float* grad, float* am, float* av, int step, float lr, float b1,
                        float b2, float eps, cudaStream_t s)
{
    const float c1 = (float)(1.0 - pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - pow((double)b2, (double)step));
    k_adam<<<ceil_div(BSPL_MLP_NPARAM, 256), 256, 0, s>>>(m->params, grad, am, av, BSPL_MLP_NPARAM, lr, b1, b2, eps,
                                                          c1, c2);
    k_sync<<<ceil_div(BSPL_MLP_NBF16, 256), 256, 0, s>>>(m->params, m->wbf16);
    return cudaGetLastError();
}

int num_sms()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

bool mlp_ok(const bspl_mlp* m) { return m && m->params && m->wbf16; }

}  // namespace

template <class Src>
cudaError_t launch_mlp_fused(const Src& src, int64_t n_max, const bspl_mlp* m, float* out, cudaStream_t s)
{
    // the shared-memory opt-in is set once per device (outside any later
    // stream capture of the calling code)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaError_t e =
            cudaFuncSetAttribute(k_mlp_fused<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmFusedBytes);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int64_t tiles = (n_max + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), (tiles + kFusedWG - 1) / kFusedWG));
    k_mlp_fused<Src><<<grid, kFusedWG * 128, kSmFusedBytes, s>>>(src, m->wbf16, m->params, out);
    return cudaGetLastError();
}

// the learned path's seed stage (query_learned.cu)
cudaError_t mlp_seed_pairs(const bspl_mlp* m, const int32_t* pq, const int32_t* ps, const float* qrec,
                           const bspl_segments* segs, int64_t cap, const unsigned long long* n_dev, float* u0,
                           cudaStream_t s)
{
    SrcPairs src{ pq, ps, qrec, segs->rec32, cap, n_dev };
    return launch_mlp_fused(src, cap, m, u0, s);
}

size_t train_ws_bytes(int64_t batch)
{
    Carver cv(nullptr, 0);
    carve_train(cv, padded(batch));
    return cv.used + 256;
}

}  // namespace bspl

using namespace bspl;

extern "C" {

bspl_status bspl_mlp_check(cudaStream_t stream)
{
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_tc_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return BSPL_ECUDA;
    if (!v) return BSPL_OK;
    if (cudaMemcpyToSymbolAsync(g_tc_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return BSPL_ECUDA;
    return BSPL_ETIMEOUT;
}

bspl_status bspl_mlp_sync(const bspl_mlp* m, cudaStream_t stream)
{
    if (!mlp_ok(m)) return BSPL_EINVAL;
    k_sync<<<ceil_div(BSPL_MLP_NBF16, 256), 256, 0, stream>>>(m->params, m->wbf16);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_forward(const bspl_mlp* m, int64_t n, const float* X, float* t, cudaStream_t stream)
{
    if (!mlp_ok(m) || n < 0 || (n > 0 && (!X || !t))) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (((uintptr_t)X & 15) != 0) return BSPL_EINVAL;
    SrcX src{ X, n };
    return launch_mlp_fused(src, n, m, t, stream) == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_features(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_seg,
                              const double* q_xyz, float* X, cudaStream_t stream)
{
    if (!segs || segs->is_surface || n < 0) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (!pair_q || !pair_seg || !q_xyz || !X || !segs->rec32 || !segs->rec64 || ((uintptr_t)X & 15)) return BSPL_EINVAL;
    k_features<<<ceil_div(n, 256), 256, 0, stream>>>(*segs, n, pair_q, pair_seg, q_xyz, X);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_labels(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_seg,
                            const double* q_xyz, float* t_star, cudaStream_t stream)
{
    if (!segs || segs->is_surface || n < 0) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (!pair_q || !pair_seg || !q_xyz || !t_star || !segs->rec64) return BSPL_EINVAL;
    k_labels<<<ceil_div(n, 128), 128, 0, stream>>>(*segs, n, pair_q, pair_seg, q_xyz, t_star);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_loss_grad(const bspl_mlp* m, int64_t n, const float* X, const float* y, float* grad,
                               float* loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!mlp_ok(m) || n < 1 || n > BSPL_MLP_MAX_BATCH || !X || !y || !grad || !loss) return BSPL_EINVAL;
    if (!ws || ws_bytes < train_ws_bytes(n)) return BSPL_EINVAL;
    const int Bp = padded(n);
    Carver cv(ws, ws_bytes);
    TrainWs w = carve_train(cv, Bp);
    if (cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return BSPL_ECUDA;
    k_gather<<<ceil_div(Bp, 256), 256, 0, stream>>>(X, y, n, 0, 1, 0, (int)n, Bp, w.Xb, w.XT, w.yb);
    cudaError_t e = batch_grad(m, w, grad, (int)n, Bp, 1.f / (float)n, loss, stream);
    return e == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_adam(const bspl_mlp* m, const float* grad, float* adam_m, float* adam_v, int32_t step, float lr,
                          float beta1, float beta2, float eps, cudaStream_t stream)
{
    if (!mlp_ok(m) || !grad || !adam_m || !adam_v || step < 1) return BSPL_EINVAL;
    return launch_adam(m, grad, adam_m, adam_v, step, lr, beta1, beta2, eps, stream) == cudaSuccess ? BSPL_OK
                                                                                                    : BSPL_ECUDA;
}

static uint64_t splitmix64(uint64_t& x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t gcd64(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

bspl_status bspl_mlp_train(const bspl_mlp* m, float* adam_m, float* adam_v, int64_t n, const float* X,
                           const float* y, int32_t epochs, int32_t batch, float lr, uint64_t seed, int32_t step0,
                           float* epoch_loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!mlp_ok(m) || !adam_m || !adam_v || n < 1 || n > 0x7fffffffLL || !X || !y || epochs < 1 || batch < 1 ||
        batch > BSPL_MLP_MAX_BATCH || !epoch_loss || step0 < 0)
        return BSPL_EINVAL;
    if (!ws || ws_bytes < train_ws_bytes(batch)) return BSPL_EINVAL;
    const int Bp = padded(batch);
    Carver cv(ws, ws_bytes);
    TrainWs w = carve_train(cv, Bp);
    if (cudaMemsetAsync(epoch_loss, 0, sizeof(float) * epochs, stream) != cudaSuccess) return BSPL_ECUDA;
    const int64_t nb = (n + batch - 1) / batch;
    const int64_t total = nb * epochs;
    uint64_t st = seed;
    int step = step0;
    for (int ep = 0; ep < epochs; ++ep) {
        uint64_t a = 1, b = 0;
        if (n > 1) {
            do a = 1 + splitmix64(st) % (uint64_t)(n - 1);
            while (gcd64(a, (uint64_t)n) != 1);
            b = splitmix64(st) % (uint64_t)n;
        }
        for (int64_t bi = 0; bi < nb; ++bi) {
            const int64_t start = bi * batch;
            const int nv = (int)std::min<int64_t>(batch, n - start);
            const int Bq = padded(nv);
            k_gather<<<ceil_div(Bq, 256), 256, 0, stream>>>(X, y, n, start, a, b, nv, Bq, w.Xb, w.XT, w.yb);
            if (batch_grad(m, w, w.grad, nv, Bq, 1.f / (float)nv / (float)nb, epoch_loss + ep, stream) != cudaSuccess)
                return BSPL_ECUDA;
            const int64_t k = (int64_t)ep * nb + bi;
            const float lr_k = lr * (1.f - 0.9f * (float)k / (float)total);
            if (launch_adam(m, w.grad, adam_m, adam_v, ++step, lr_k, 0.9f, 0.999f, 1e-8f, stream) != cudaSuccess)
                return BSPL_ECUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // extern "C"
