// Learned Newton seed: the small MLP of bspl_mlp.h on the tensor cores.
//
// Inference (k_mlp_fused): one persistent block per SM of four warpgroups.
// The BF16 weights of the three 128-wide layers stay in shared memory; each
// warpgroup runs its own tiles of 128 rows: inputs -> shared memory (BF16) ->
// tcgen05.mma into its 128 tensor-memory columns -> tcgen05.ld, bias, GELU
// (packed BF16 arithmetic, two columns per instruction) -> shared memory ->
// next layer; the last layer's epilogue also takes
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
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s bound on every mbarrier wait

// Shape of a seed network IN -> 128 -> 128 -> 128 -> OUT: offsets of its
// tensors in the FP32 parameter vector and in the BF16 copy the kernels read
// (W1, W2, W3, W2^T, W3^T, W4).
template <int IN_, int OUT_>
struct Net {
    static constexpr int IN = IN_, OUT = OUT_;
    static constexpr int W1 = 0, B1 = kH * IN, W2 = B1 + kH, B2 = W2 + kH * kH, W3 = B2 + kH, B3 = W3 + kH * kH,
                         W4 = B3 + kH, B4 = W4 + OUT * kH, NPARAM = (B4 + OUT + 3) / 4 * 4;
    static constexpr int BW1 = 0, BW2 = kH * IN, BW3 = BW2 + kH * kH, BW2T = BW3 + kH * kH, BW3T = BW2T + kH * kH,
                         BW4 = BW3T + kH * kH, NBF16 = BW4 + OUT * kH;
};
using CurveNet = Net<BSPL_MLP_IN, 1>;
using SurfNet = Net<BSPL_SMLP_IN, BSPL_SMLP_OUT>;
static_assert(CurveNet::B1 == BSPL_MLP_OFF_B1 && CurveNet::W2 == BSPL_MLP_OFF_W2 && CurveNet::B2 == BSPL_MLP_OFF_B2 &&
                  CurveNet::W3 == BSPL_MLP_OFF_W3 && CurveNet::B3 == BSPL_MLP_OFF_B3 &&
                  CurveNet::W4 == BSPL_MLP_OFF_W4 && CurveNet::B4 == BSPL_MLP_OFF_B4 &&
                  CurveNet::NPARAM == BSPL_MLP_NPARAM && CurveNet::NBF16 == BSPL_MLP_NBF16,
              "curve network layout");
static_assert(SurfNet::B1 == BSPL_SMLP_OFF_B1 && SurfNet::W2 == BSPL_SMLP_OFF_W2 && SurfNet::B2 == BSPL_SMLP_OFF_B2 &&
                  SurfNet::W3 == BSPL_SMLP_OFF_W3 && SurfNet::B3 == BSPL_SMLP_OFF_B3 &&
                  SurfNet::W4 == BSPL_SMLP_OFF_W4 && SurfNet::B4 == BSPL_SMLP_OFF_B4 &&
                  SurfNet::NPARAM == BSPL_SMLP_NPARAM && SurfNet::NBF16 == BSPL_SMLP_NBF16,
              "surface network layout");

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
template <class N>
__global__ void k_sync(const float* __restrict__ p, uint16_t* __restrict__ w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N::NBF16) return;
    float v;
    if (i < N::BW2) v = p[N::W1 + i];
    else if (i < N::BW3) v = p[N::W2 + (i - N::BW2)];
    else if (i < N::BW2T) v = p[N::W3 + (i - N::BW3)];
    else if (i < N::BW3T) {
        int j = i - N::BW2T, r = j / kH, c = j % kH;  // W2^T[r][c] = W2[c][r]
        v = p[N::W2 + c * kH + r];
    } else if (i < N::BW4) {
        int j = i - N::BW3T, r = j / kH, c = j % kH;
        v = p[N::W3 + c * kH + r];
    } else v = p[N::W4 + (i - N::BW4)];
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

template <class N>
struct SrcX {
    using Shape = N;
    const float* X;
    int64_t n;
    __device__ int64_t count() const { return n; }
    // row i's inputs are contiguous: nothing to fetch ahead
    __device__ int2 ahead_index(int64_t) const { return make_int2(0, 0); }
    __device__ void ahead_fetch(int2) const {}
    __device__ void features(int64_t i, float* f) const
    {
        const float4* p = reinterpret_cast<const float4*>(X + N::IN * i);
#pragma unroll
        for (int k = 0; k < N::IN / 4; ++k) {
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
    using Shape = Net<BSPL_MLP_IN, 1>;
    const int32_t* pq;  // sorted query position
    const int32_t* ps;
    const float* qrec;  // per sorted query: q hi[3], q lo[3], ...
    const float* rec32;
    int64_t cap;
    const unsigned long long* n_dev;
    __device__ int64_t count() const { return min(cap, (int64_t)*n_dev); }
    // the records row i gathers, fetched into L2 one tile ahead: the indices
    // are loaded early, the prefetches issued once they have arrived
    __device__ int2 ahead_index(int64_t i) const { return make_int2(ps[i], pq[i]); }
    __device__ void ahead_fetch(int2 ix) const
    {
        const float* r = rec32 + (int64_t)BSPL_CREC32 * ix.x;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(r));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(r + 16));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(qrec + 8 * (int64_t)ix.y));
    }
    __device__ void features(int64_t i, float* f) const
    {
        pair_features(rec32 + (int64_t)BSPL_CREC32 * ps[i], qrec + 8 * (int64_t)pq[i], f);
    }
};

// Inputs of a (query, patch) pair for the surface network (bspl_mlp.h): the
// bicubic's control points relative to P00 from its FP32 power coefficients
// a_kl (P_ij - P00 = sum over (k, l) != (0, 0) of T_ik T_jl a_kl with the
// power-to-Bernstein matrix T_ik = C(i, k) / C(3, k), Sec. 4.3), in the
// frame of their box; the query q - P00 formed in FP64 by the caller (qm).
__device__ __forceinline__ void patch_features(const float* __restrict__ r32, const float qm[3], float* f)
{
    const float T[4][4] = { { 1.f, 0.f, 0.f, 0.f },
                            { 1.f, 1.f / 3.f, 0.f, 0.f },
                            { 1.f, 2.f / 3.f, 1.f / 3.f, 0.f },
                            { 1.f, 1.f, 1.f, 1.f } };
    const float* a = r32 + 6;
    float lo[3] = { 0.f, 0.f, 0.f }, hi[3] = { 0.f, 0.f, 0.f };
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float d = 0.f;
#pragma unroll
                for (int k = 0; k <= i; ++k)
#pragma unroll
                    for (int l = 0; l <= j; ++l)
                        if (k | l) d = fmaf(T[i][k] * T[j][l], a[(k * 4 + l) * 3 + c], d);
                f[(i * 4 + j) * 3 + c] = d;
                lo[c] = fminf(lo[c], d);
                hi[c] = fmaxf(hi[c], d);
            }
    float cc[3], ext = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cc[c] = 0.5f * (lo[c] + hi[c]);
        ext = fmaxf(ext, hi[c] - lo[c]);
    }
    const float s = ext > 0.f ? 1.f / ext : 1.f;
    // frame: e1 along P30 - P00, e2 the part of P03 - P00 across e1, n = e1 x e2
    float e1[3], e2[3], nn[3], v[3];
    float l1 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e1[c] = f[(3 * 4 + 0) * 3 + c];
        l1 += e1[c] * e1[c];
    }
    l1 = sqrtf(l1);
#pragma unroll
    for (int c = 0; c < 3; ++c) e1[c] = l1 > 0.f ? e1[c] / l1 : (c == 0 ? 1.f : 0.f);
    float pr = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) pr += f[(0 * 4 + 3) * 3 + c] * e1[c];
    float l2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e2[c] = f[(0 * 4 + 3) * 3 + c] - pr * e1[c];
        l2 += e2[c] * e2[c];
    }
    l2 = sqrtf(l2);
    if (l2 > 0.f) {
#pragma unroll
        for (int c = 0; c < 3; ++c) e2[c] /= l2;
    } else {
        // any unit vector across e1
        const int ax = fabsf(e1[0]) < 0.9f ? 0 : 1;
        float t[3] = { 0.f, 0.f, 0.f };
        t[ax] = 1.f;
        const float d = t[0] * e1[0] + t[1] * e1[1] + t[2] * e1[2];
        float l = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e2[c] = t[c] - d * e1[c];
            l += e2[c] * e2[c];
        }
        l = sqrtf(l);
#pragma unroll
        for (int c = 0; c < 3; ++c) e2[c] /= l;
    }
    nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = (qm[c] - cc[c]) * s;
    const float a1 = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
    const float a2 = v[0] * e2[0] + v[1] * e2[1] + v[2] * e2[2];
    const float a3 = fminf(fmaxf(v[0] * nn[0] + v[1] * nn[1] + v[2] * nn[2], -1.f), 1.f);
#pragma unroll
    for (int k = 0; k < 48; ++k) f[k] = (f[k] - cc[k % 3]) * s;
#pragma unroll
    for (int c = 0; c < 3; ++c) f[48 + c] = a1 * e1[c] + a2 * e2[c] + a3 * nn[c];
#pragma unroll
    for (int k = 51; k < 64; ++k) f[k] = 0.f;
}

// the learned surface path's pairs [0, min(cap, *n_dev)) of (sorted query
// position, patch)
struct SrcSurfPairs {
    using Shape = Net<BSPL_SMLP_IN, BSPL_SMLP_OUT>;
    const int32_t* pq;     // sorted query position
    const int32_t* pp;     // patch
    const int32_t* order;  // sorted position -> query index
    const double* q_xyz;
    const float* rec32;
    const double* rec64;
    int64_t cap;
    const unsigned long long* n_dev;
    __device__ int64_t count() const { return min(cap, (int64_t)*n_dev); }
    __device__ int2 ahead_index(int64_t i) const { return make_int2(pp[i], 0); }
    __device__ void ahead_fetch(int2 ix) const
    {
        const float* r = rec32 + (int64_t)BSPL_SREC32 * ix.x;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(r));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(r + 32));
    }
    __device__ void features(int64_t i, float* f) const
    {
        const int64_t p = pp[i];
        const double* q = q_xyz + 3 * (int64_t)order[pq[i]];
        const double* a00 = rec64 + (int64_t)BSPL_SREC64 * p + 6;
        const float qm[3] = { (float)(q[0] - a00[0]), (float)(q[1] - a00[1]), (float)(q[2] - a00[2]) };
        patch_features(rec32 + (int64_t)BSPL_SREC32 * p, qm, f);
    }
};

namespace {

// ------------------------------------------------------- fused inference
constexpr int kFusedWG = 4;  // warpgroups per block

// shared-memory layout of the fused kernel for network N: W1 [128][IN],
// W2, W3 in the core-matrix layout; biases, W4 and b4 as FP32; one 32 KB
// activation tile per warpgroup (a tile's features are staged there too:
// they are consumed by the first MMA before its epilogue overwrites them);
// the mbarriers
template <class N>
struct FusedSmem {
    static constexpr int W1 = 0, W2 = kH * N::IN * 2, W3 = W2 + kH * kH * 2, BIAS = W3 + kH * kH * 2;
    static constexpr int BIAS_BYTES = ((3 * kH + N::OUT * kH + N::OUT) * 4 + 127) / 128 * 128;
    static constexpr int X = BIAS + BIAS_BYTES, BAR = X + kFusedWG * kH * kH * 2, BYTES = BAR + 64;
    static_assert(BYTES <= 227 * 1024, "fused kernel shared memory");
};

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
            pk[j] = tc::gelu_bf16x2(v[2 * j] + b[cb * 32 + 2 * j], v[2 * j + 1] + b[cb * 32 + 2 * j + 1]);
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
    using N = typename Src::Shape;
    using L = FusedSmem<N>;
    extern __shared__ __align__(1024) uint8_t sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::BAR + 8 * kFusedWG);
    volatile int* okf = reinterpret_cast<volatile int*>(sm + L::BAR + 8 * kFusedWG + 8);
    float* bias = reinterpret_cast<float*>(sm + L::BIAS);
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
    stage_weights(sm + L::W1, wb + N::BW1, kH, N::IN, tid, blockDim.x);
    stage_weights(sm + L::W2, wb + N::BW2, kH, kH, tid, blockDim.x);
    stage_weights(sm + L::W3, wb + N::BW3, kH, kH, tid, blockDim.x);
    for (int i = tid; i < 3 * kH; i += blockDim.x) {
        const int l = i / kH, c = i % kH;
        const int off = l == 0 ? N::B1 : (l == 1 ? N::B2 : N::B3);
        bias[i] = params[off + c];
    }
    for (int i = tid; i < N::OUT * kH; i += blockDim.x) bias[3 * kH + i] = bf2f(wb[N::BW4 + i]);
    if (tid < N::OUT) bias[3 * kH + N::OUT * kH + tid] = params[N::B4 + tid];
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t tacc = *tslot + (uint32_t)(g * 128);
    const uint32_t tl = tacc + ((uint32_t)((warp & 3) * 32) << 16);
    uint8_t* X = sm + L::X + g * kH * kH * 2;
    const uint32_t aX = tc::smem_u32(X);
    const uint32_t aW1 = tc::smem_u32(sm + L::W1), aW2 = tc::smem_u32(sm + L::W2), aW3 = tc::smem_u32(sm + L::W3);
    constexpr uint32_t idesc = tc::idesc_bf16(128, kH);
    const float* w4 = bias + 3 * kH;
    const float* b4 = bias + 3 * kH + N::OUT * kH;
    const int bar_id = 1 + g;
    uint32_t phase = 0;

    const int64_t n = src.count();
    const int64_t ntiles = (n + 127) / 128;
    // one MMA group, completion awaited by the issuing thread, result shared
    auto run_layer = [&](int layer) -> bool {
        if (r == 0) {
            tc::fence_after_sync();
            if (layer == 0) {
#pragma unroll
                for (int ks = 0; ks < N::IN / 16; ++ks)
                    tc::mma_bf16(tacc, tc::sdesc(aX + ks * 256, 128, N::IN * 16),
                                 tc::sdesc(aW1 + ks * 256, 128, N::IN * 16), idesc, ks > 0);
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

    const int64_t tstride = (int64_t)gridDim.x * kFusedWG;
    for (int64_t tile = (int64_t)blockIdx.x * kFusedWG + g; tile < ntiles; tile += tstride) {
        const int64_t i = tile * 128 + r;
        // the next tile's row: its indices now, its records into L2 below
        const int64_t inext = i + tstride * 128;
        const int2 ahead = inext < n ? src.ahead_index(inext) : make_int2(-1, -1);
        {
            float f[N::IN];
            if (i < n) src.features(i, f);
            else {
#pragma unroll
                for (int k = 0; k < N::IN; ++k) f[k] = 0.f;
            }
            // this row's features, BF16, into the tile's activation buffer
#pragma unroll
            for (int kg = 0; kg < N::IN / 8; ++kg)
                *reinterpret_cast<uint4*>(X + (r >> 3) * N::IN * 16 + kg * 128 + (r & 7) * 16) =
                    make_uint4(tc::pack_bf16(f[8 * kg], f[8 * kg + 1]), tc::pack_bf16(f[8 * kg + 2], f[8 * kg + 3]),
                               tc::pack_bf16(f[8 * kg + 4], f[8 * kg + 5]),
                               tc::pack_bf16(f[8 * kg + 6], f[8 * kg + 7]));
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        named_sync(bar_id, 128);
        if (ahead.x >= 0) src.ahead_fetch(ahead);
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
        float z[N::OUT];
#pragma unroll
        for (int o = 0; o < N::OUT; ++o) z[o] = b4[o];
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
            float v[32];
            tc::tmem_ld32(tl + cb * 32, v);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
                const int c = cb * 32 + j;
                const uint32_t hp = tc::gelu_bf16x2(v[j] + bias[2 * kH + c], v[j + 1] + bias[2 * kH + c + 1]);
                const float h0 = __uint_as_float(hp << 16), h1 = __uint_as_float(hp & 0xffff0000u);
#pragma unroll
                for (int o = 0; o < N::OUT; ++o) z[o] = fmaf(h1, w4[o * kH + c + 1], fmaf(h0, w4[o * kH + c], z[o]));
            }
        }
        if (i < n) {
#pragma unroll
            for (int o = 0; o < N::OUT; ++o) out[N::OUT * i + o] = 1.f / (1.f + __expf(-z[o]));
        }
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
template <class N>
__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ y, int64_t n, int64_t start,
                         uint64_t a, uint64_t b, int nvalid, int Bp, uint16_t* __restrict__ Xb,
                         uint16_t* __restrict__ XT, float* __restrict__ yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp) return;
    int64_t j = -1;
    if (i < nvalid) {
        const uint64_t x = (uint64_t)(start + i) % (uint64_t)n;
        j = (int64_t)((a * x % (uint64_t)n + b) % (uint64_t)n);
    }
#pragma unroll 4
    for (int k = 0; k < N::IN; ++k) {
        const uint16_t h = f2bf(j >= 0 ? X[N::IN * j + k] : 0.f);
        Xb[N::IN * i + k] = h;
        XT[(int64_t)k * Bp + i] = h;
    }
#pragma unroll
    for (int o = 0; o < N::OUT; ++o) yb[N::OUT * i + o] = j >= 0 ? y[N::OUT * j + o] : 0.f;
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

// output layer: z4 = H3 W4^T + b4, t = sigmoid, loss, dz4 (one warp per row);
// the loss is the mean over rows and outputs: inv = 1 / (nvalid OUT)
template <class N>
__global__ void k_head(const uint16_t* __restrict__ H3, const uint16_t* __restrict__ wb,
                       const float* __restrict__ params, const float* __restrict__ yb, int nvalid, int Bp,
                       float inv, float loss_scale, float* __restrict__ dz4, float* __restrict__ loss)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= Bp) return;
#pragma unroll
    for (int o = 0; o < N::OUT; ++o) {
        float z = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = lane + 32 * k;
            z += bf2f(H3[(int64_t)row * kH + c]) * bf2f(wb[N::BW4 + o * kH + c]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) z += __shfl_xor_sync(0xffffffffu, z, off);
        if (lane == 0) {
            z += params[N::B4 + o];
            const float t = 1.f / (1.f + __expf(-z));
            float d = 0.f;
            if (row < nvalid) {
                const float rr = t - yb[N::OUT * row + o];
                d = 2.f * inv * rr * t * (1.f - t);
                atomicAdd(loss, rr * rr * loss_scale);
            }
            dz4[N::OUT * row + o] = d;
        }
    }
}

// dZ = dH (.) GELU'(Z) with dH = dz4 W4 (head) or the GEMM output; writes
// BF16 dZ and its transpose; column sums of dZ -> bias gradient; for the
// head also the W4 and b4 gradients
template <class N, bool HEAD>
__global__ void k_act_back(const float* __restrict__ dH, const float* __restrict__ dz4,
                           const uint16_t* __restrict__ H3, const uint16_t* __restrict__ wb,
                           const float* __restrict__ Z, uint16_t* __restrict__ dZb, uint16_t* __restrict__ dZT,
                           float* __restrict__ gbias, float* __restrict__ gw4, float* __restrict__ gb4, int Bp)
{
    __shared__ uint16_t tile[32][33];
    __shared__ float csum[8][32], cw4[N::OUT][8][32], cb4[N::OUT][8];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float sb = 0.f, sw[N::OUT], s4[N::OUT];
#pragma unroll
    for (int o = 0; o < N::OUT; ++o) sw[o] = s4[o] = 0.f;
    for (int k = ty; k < 32; k += blockDim.y) {
        const int row = r0 + k, col = c0 + tx;
        const int64_t idx = (int64_t)row * kH + col;
        float g = 0.f;
        if (HEAD) {
            const float h3 = bf2f(H3[idx]);
#pragma unroll
            for (int o = 0; o < N::OUT; ++o) {
                const float d4 = dz4[N::OUT * row + o];
                g += d4 * bf2f(wb[N::BW4 + o * kH + col]);
                sw[o] += d4 * h3;
                if (tx == 0) s4[o] += d4;
            }
        } else g = dH[idx];
        const float dz = g * tc::gelu_grad(Z[idx]);
        sb += dz;
        const uint16_t h = f2bf(dz);
        dZb[idx] = h;
        tile[k][tx] = h;
    }
    csum[ty][tx] = sb;
#pragma unroll
    for (int o = 0; o < N::OUT; ++o) {
        cw4[o][ty][tx] = sw[o];
        if (tx == 0) cb4[o][ty] = s4[o];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += blockDim.y) dZT[(int64_t)(c0 + k) * Bp + r0 + tx] = tile[tx][k];
    if (ty == 0) {
        float a = 0.f;
        for (int k = 0; k < (int)blockDim.y; ++k) a += csum[k][tx];
        atomicAdd(gbias + c0 + tx, a);
        if (HEAD) {
#pragma unroll
            for (int o = 0; o < N::OUT; ++o) {
                float w = 0.f;
                for (int k = 0; k < (int)blockDim.y; ++k) w += cw4[o][k][tx];
                atomicAdd(gw4 + o * kH + c0 + tx, w);
                if (tx == 0 && blockIdx.y == 0) {
                    float t = 0.f;
                    for (int k = 0; k < (int)blockDim.y; ++k) t += cb4[o][k];
                    atomicAdd(gb4 + o, t);
                }
            }
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

// ------------------------------------------------ surface network inputs
__global__ void k_smlp_features(const bspl_segments S, int64_t n, const int32_t* __restrict__ pq,
                                const int32_t* __restrict__ pp, const double* __restrict__ q_xyz, float* __restrict__ X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float f[BSPL_SMLP_IN];
    const int64_t p = pp[i];
    if (p < 0 || p >= S.capacity || pq[i] < 0) {
#pragma unroll
        for (int k = 0; k < BSPL_SMLP_IN; ++k) f[k] = __int_as_float(0x7fc00000);
    } else {
        const double* q = q_xyz + 3 * (int64_t)pq[i];
        const double* a00 = S.rec64 + (int64_t)BSPL_SREC64 * p + 6;
        const float qm[3] = { (float)(q[0] - a00[0]), (float)(q[1] - a00[1]), (float)(q[2] - a00[2]) };
        patch_features(S.rec32 + (int64_t)BSPL_SREC32 * p, qm, f);
    }
    float4* o = reinterpret_cast<float4*>(X + BSPL_SMLP_IN * i);
#pragma unroll
    for (int k = 0; k < BSPL_SMLP_IN / 4; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

// D = |S(u,v) - q|^2 of a bicubic in power form (a[(i*4+j)*3+c], the
// constant term already minus q), its gradient g and Hessian h (halved)
template <class R>
__device__ __forceinline__ R bicubic_dgh(const R* a, R u, R v, R* g, R* h)
{
    R D = 0;
    if (g) g[0] = g[1] = h[0] = h[1] = h[2] = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R s = 0, su = 0, sv = 0, suu = 0, suv = 0, svv = 0;
#pragma unroll
        for (int i = 3; i >= 0; --i) {
            R p = 0, p1 = 0, p2 = 0;
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                p2 = p2 * v + R(2) * p1;
                p1 = p1 * v + p;
                p = p * v + a[(i * 4 + j) * 3 + c];
            }
            suu = suu * u + R(2) * su;
            suv = suv * u + sv;
            su = su * u + s;
            s = s * u + p;
            svv = svv * u + p2;
            sv = sv * u + p1;
        }
        D += s * s;
        if (g) {
            g[0] += s * su;
            g[1] += s * sv;
            h[0] += su * su + s * suu;
            h[1] += su * sv + s * suv;
            h[2] += sv * sv + s * svv;
        }
    }
    return D;
}

// projected Newton with halving on [0,1]^2 (gradient step where the Hessian
// is not positive definite), FP64
__device__ double patch_newton64(const double* a, double& u, double& v)
{
    double g[2], h[3];
    double D = bicubic_dgh<double>(a, u, v, g, h);
    for (int it = 0; it < 60; ++it) {
        const bool fu = !((u <= 0.0 && g[0] > 0.0) || (u >= 1.0 && g[0] < 0.0));
        const bool fv = !((v <= 0.0 && g[1] > 0.0) || (v >= 1.0 && g[1] < 0.0));
        double su = 0.0, sv = 0.0;
        const double det = h[0] * h[2] - h[1] * h[1];
        if (fu && fv && h[0] > 0.0 && det > 0.0) {
            su = -(h[2] * g[0] - h[1] * g[1]) / det;
            sv = -(h[0] * g[1] - h[1] * g[0]) / det;
        } else {
            if (fu) su = h[0] > 0.0 ? -g[0] / h[0] : -g[0];
            if (fv) sv = h[2] > 0.0 ? -g[1] / h[2] : -g[1];
        }
        if (su == 0.0 && sv == 0.0) break;
        double lam = 1.0, un = u, vn = v, Dn = D;
        bool acc = false;
        for (int ls = 0; ls < 40; ++ls) {
            un = fmin(fmax(u + lam * su, 0.0), 1.0);
            vn = fmin(fmax(v + lam * sv, 0.0), 1.0);
            Dn = bicubic_dgh<double>(a, un, vn, nullptr, nullptr);
            if (Dn <= D) {
                acc = true;
                break;
            }
            lam *= 0.5;
        }
        if (!acc) break;
        const double step = fabs(un - u) + fabs(vn - v);
        u = un;
        v = vn;
        D = bicubic_dgh<double>(a, u, v, g, h);
        if (step <= 1e-15) break;
    }
    return D;
}

__global__ void k_smlp_labels(const bspl_segments S, int64_t n, const int32_t* __restrict__ pq,
                              const int32_t* __restrict__ pp, const double* __restrict__ q_xyz, float* __restrict__ uv)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = pp[i];
    if (p < 0 || p >= S.capacity || pq[i] < 0) {
        uv[2 * i] = uv[2 * i + 1] = __int_as_float(0x7fc00000);
        return;
    }
    const double* q = q_xyz + 3 * (int64_t)pq[i];
    const double* a64 = S.rec64 + (int64_t)BSPL_SREC64 * p + 6;
    const float* a32 = S.rec32 + (int64_t)BSPL_SREC32 * p + 6;
    float af[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) af[k] = a32[k];
    for (int c = 0; c < 3; ++c) af[c] = (float)(a64[c] - q[c]);
    // 17 x 17 FP32 samples: the two smallest
    float d0 = INFINITY, d1 = INFINITY;
    int k0 = 0, k1 = 0;
    for (int k = 0; k < 17 * 17; ++k) {
        const float u = (float)(k / 17) * (1.f / 16.f), v = (float)(k % 17) * (1.f / 16.f);
        const float D = bicubic_dgh<float>(af, u, v, nullptr, nullptr);
        if (D < d0) {
            d1 = d0;
            k1 = k0;
            d0 = D;
            k0 = k;
        } else if (D < d1) {
            d1 = D;
            k1 = k;
        }
    }
    double a[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) a[k] = a64[k];
    for (int c = 0; c < 3; ++c) a[c] -= q[c];
    double bu = 0.0, bv = 0.0, bD = INFINITY;
    for (int t = 0; t < 2; ++t) {
        const int k = t ? k1 : k0;
        double u = (double)(k / 17) / 16.0, v = (double)(k % 17) / 16.0;
        const double D = patch_newton64(a, u, v);
        if (D < bD || (D == bD && (u < bu || (u == bu && v < bv)))) {
            bD = D;
            bu = u;
            bv = v;
        }
    }
    uv[2 * i] = (float)bu;
    uv[2 * i + 1] = (float)bv;
}

// workspace of one training batch of Bp rows (multiple of 128)
struct TrainWs {
    uint16_t *Xb, *XT, *H1, *H2, *H3, *H1T, *H2T, *dZb, *dZT;
    float *yb, *Z1, *Z2, *Z3, *dz4, *dH, *grad, *loss;
};

template <class N>
TrainWs carve_train(Carver& cv, int Bp)
{
    TrainWs w{};
    w.Xb = cv.take<uint16_t>((size_t)Bp * N::IN);
    w.XT = cv.take<uint16_t>((size_t)Bp * N::IN);
    w.yb = cv.take<float>((size_t)Bp * N::OUT);
    w.Z1 = cv.take<float>((size_t)Bp * kH);
    w.Z2 = cv.take<float>((size_t)Bp * kH);
    w.Z3 = cv.take<float>((size_t)Bp * kH);
    w.H1 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H2 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H3 = cv.take<uint16_t>((size_t)Bp * kH);
    w.H1T = cv.take<uint16_t>((size_t)Bp * kH);
    w.H2T = cv.take<uint16_t>((size_t)Bp * kH);
    w.dz4 = cv.take<float>((size_t)Bp * N::OUT);
    w.dH = cv.take<float>((size_t)Bp * kH);
    w.dZb = cv.take<uint16_t>((size_t)Bp * kH);
    w.dZT = cv.take<uint16_t>((size_t)Bp * kH);
    w.grad = cv.take<float>(N::NPARAM);
    w.loss = cv.take<float>(4);
    return w;
}

int padded(int64_t batch) { return (int)((batch + 127) / 128 * 128); }

// forward + backward of one padded batch already gathered into w (Xb, XT,
// yb); grad overwritten, loss_scale * sum of squared residuals added to *loss
template <class N>
cudaError_t batch_grad(const bspl_mlp* m, const TrainWs& w, float* grad, int nvalid, int Bp, float loss_scale,
                       float* loss, cudaStream_t s)
{
    const uint16_t* wb = m->wbf16;
    const float* p = m->params;
    float* g = grad;
    cudaError_t e = cudaMemsetAsync(g, 0, sizeof(float) * N::NPARAM, s);
    if (e != cudaSuccess) return e;
    const dim3 tb(32, 8), tg(Bp / 32, kH / 32);
    const int splits = std::max(1, Bp / 512);
    // forward: Z_l = H_{l-1} W_l^T + b_l, H_l = GELU(Z_l)
    if ((e = gemm_nt(w.Xb, N::IN, wb + N::BW1, N::IN, w.Z1, kH, Bp, kH, N::IN, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z1, p + N::B1, w.H1, w.H1T, Bp);
    if ((e = gemm_nt(w.H1, kH, wb + N::BW2, kH, w.Z2, kH, Bp, kH, kH, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z2, p + N::B2, w.H2, w.H2T, Bp);
    if ((e = gemm_nt(w.H2, kH, wb + N::BW3, kH, w.Z3, kH, Bp, kH, kH, 1, false, s))) return e;
    k_bias_act<<<tg, tb, 0, s>>>(w.Z3, p + N::B3, w.H3, nullptr, Bp);
    k_head<N><<<Bp / 8, 256, 0, s>>>(w.H3, wb, p, w.yb, nvalid, Bp, 1.f / ((float)nvalid * N::OUT),
                                     loss_scale / N::OUT, w.dz4, loss);
    // layer 3: dZ3 = (dz4 W4) (.) GELU'(Z3); dW3 = dZ3^T H2; dH2 = dZ3 W3
    k_act_back<N, true><<<tg, tb, 0, s>>>(nullptr, w.dz4, w.H3, wb, w.Z3, w.dZb, w.dZT, g + N::B3, g + N::W4,
                                          g + N::B4, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.H2T, Bp, g + N::W3, kH, kH, kH, Bp, splits, true, s))) return e;
    if ((e = gemm_nt(w.dZb, kH, wb + N::BW3T, kH, w.dH, kH, Bp, kH, kH, 1, false, s))) return e;
    // layer 2
    k_act_back<N, false><<<tg, tb, 0, s>>>(w.dH, nullptr, nullptr, wb, w.Z2, w.dZb, w.dZT, g + N::B2, nullptr,
                                           nullptr, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.H1T, Bp, g + N::W2, kH, kH, kH, Bp, splits, true, s))) return e;
    if ((e = gemm_nt(w.dZb, kH, wb + N::BW2T, kH, w.dH, kH, Bp, kH, kH, 1, false, s))) return e;
    // layer 1: dW1 = dZ1^T X (N = IN columns)
    k_act_back<N, false><<<tg, tb, 0, s>>>(w.dH, nullptr, nullptr, wb, w.Z1, w.dZb, w.dZT, g + N::B1, nullptr,
                                           nullptr, Bp);
    if ((e = gemm_nt(w.dZT, Bp, w.XT, Bp, g + N::W1, N::IN, kH, N::IN, Bp, splits, true, s))) return e;
    return cudaGetLastError();
}

template <class N>
cudaError_t launch_adam(const bspl_mlp* m, const float* grad, float* am, float* av, int step, float lr, float b1,
                        float b2, float eps, cudaStream_t s)
{
    const float c1 = (float)(1.0 - pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - pow((double)b2, (double)step));
    k_adam<<<ceil_div(N::NPARAM, 256), 256, 0, s>>>(m->params, grad, am, av, N::NPARAM, lr, b1, b2, eps, c1, c2);
    k_sync<N><<<ceil_div(N::NBF16, 256), 256, 0, s>>>(m->params, m->wbf16);
    return cudaGetLastError();
}

int num_sms()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

bool mlp_ok(const bspl_mlp* m)
{
    return m && m->params && m->wbf16 && (m->kind == BSPL_MLP_CURVE || m->kind == BSPL_MLP_SURFACE);
}

}  // namespace

template <class Src>
cudaError_t launch_mlp_fused(const Src& src, int64_t n_max, const bspl_mlp* m, float* out, cudaStream_t s)
{
    // the shared-memory opt-in is set once per device (outside any later
    // stream capture of the calling code)
    constexpr int bytes = FusedSmem<typename Src::Shape>::BYTES;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_fused<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int64_t tiles = (n_max + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), (tiles + kFusedWG - 1) / kFusedWG));
    k_mlp_fused<Src><<<grid, kFusedWG * 128, bytes, s>>>(src, m->wbf16, m->params, out);
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

// the learned surface path's seed stage (query_surfaces.cu): (u, v) of every
// pair [0, min(cap, *n_dev)), two floats per pair
cudaError_t mlp_seed_surface_pairs(const bspl_mlp* m, const int32_t* pq, const int32_t* pp, const int32_t* order,
                                   const double* q_xyz, const bspl_segments* segs, int64_t cap,
                                   const unsigned long long* n_dev, float* uv0, cudaStream_t s)
{
    SrcSurfPairs src{ pq, pp, order, q_xyz, segs->rec32, segs->rec64, cap, n_dev };
    return launch_mlp_fused(src, cap, m, uv0, s);
}

size_t train_ws_bytes(int kind, int64_t batch)
{
    Carver cv(nullptr, 0);
    if (kind == BSPL_MLP_SURFACE) carve_train<SurfNet>(cv, padded(batch));
    else carve_train<CurveNet>(cv, padded(batch));
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
    if (m->kind == BSPL_MLP_SURFACE)
        k_sync<SurfNet><<<ceil_div(SurfNet::NBF16, 256), 256, 0, stream>>>(m->params, m->wbf16);
    else
        k_sync<CurveNet><<<ceil_div(CurveNet::NBF16, 256), 256, 0, stream>>>(m->params, m->wbf16);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_forward(const bspl_mlp* m, int64_t n, const float* X, float* t, cudaStream_t stream)
{
    if (!mlp_ok(m) || n < 0 || (n > 0 && (!X || !t))) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (((uintptr_t)X & 15) != 0) return BSPL_EINVAL;
    cudaError_t e;
    if (m->kind == BSPL_MLP_SURFACE) e = launch_mlp_fused(SrcX<SurfNet>{ X, n }, n, m, t, stream);
    else e = launch_mlp_fused(SrcX<CurveNet>{ X, n }, n, m, t, stream);
    return e == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
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

extern "C++" template <class N>
bspl_status loss_grad_impl(const bspl_mlp* m, int64_t n, const float* X, const float* y, float* grad,
                                  float* loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    const int Bp = padded(n);
    Carver cv(ws, ws_bytes);
    TrainWs w = carve_train<N>(cv, Bp);
    if (cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return BSPL_ECUDA;
    k_gather<N><<<ceil_div(Bp, 256), 256, 0, stream>>>(X, y, n, 0, 1, 0, (int)n, Bp, w.Xb, w.XT, w.yb);
    cudaError_t e = batch_grad<N>(m, w, grad, (int)n, Bp, 1.f / (float)n, loss, stream);
    return e == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_loss_grad(const bspl_mlp* m, int64_t n, const float* X, const float* y, float* grad,
                               float* loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!mlp_ok(m) || n < 1 || n > BSPL_MLP_MAX_BATCH || !X || !y || !grad || !loss) return BSPL_EINVAL;
    if (!ws || ws_misaligned(ws) || ws_bytes < train_ws_bytes(m->kind, n)) return BSPL_EINVAL;
    if (m->kind == BSPL_MLP_SURFACE) return loss_grad_impl<SurfNet>(m, n, X, y, grad, loss, ws, ws_bytes, stream);
    return loss_grad_impl<CurveNet>(m, n, X, y, grad, loss, ws, ws_bytes, stream);
}

bspl_status bspl_mlp_adam(const bspl_mlp* m, const float* grad, float* adam_m, float* adam_v, int32_t step, float lr,
                          float beta1, float beta2, float eps, cudaStream_t stream)
{
    if (!mlp_ok(m) || !grad || !adam_m || !adam_v || step < 1) return BSPL_EINVAL;
    const cudaError_t e = m->kind == BSPL_MLP_SURFACE
                              ? launch_adam<SurfNet>(m, grad, adam_m, adam_v, step, lr, beta1, beta2, eps, stream)
                              : launch_adam<CurveNet>(m, grad, adam_m, adam_v, step, lr, beta1, beta2, eps, stream);
    return e == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_smlp_features(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_patch,
                               const double* q_xyz, float* X, cudaStream_t stream)
{
    if (!segs || !segs->is_surface || n < 0) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (!pair_q || !pair_patch || !q_xyz || !X || !segs->rec32 || !segs->rec64 || ((uintptr_t)X & 15))
        return BSPL_EINVAL;
    k_smlp_features<<<ceil_div(n, 128), 128, 0, stream>>>(*segs, n, pair_q, pair_patch, q_xyz, X);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_smlp_labels(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_patch,
                             const double* q_xyz, float* uv, cudaStream_t stream)
{
    if (!segs || !segs->is_surface || n < 0) return BSPL_EINVAL;
    if (n == 0) return BSPL_OK;
    if (!pair_q || !pair_patch || !q_xyz || !uv || !segs->rec32 || !segs->rec64) return BSPL_EINVAL;
    k_smlp_labels<<<ceil_div(n, 128), 128, 0, stream>>>(*segs, n, pair_q, pair_patch, q_xyz, uv);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
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

extern "C++" template <class N>
bspl_status train_impl(const bspl_mlp* m, float* adam_m, float* adam_v, int64_t n, const float* X,
                              const float* y, int32_t epochs, int32_t batch, float lr, uint64_t seed, int32_t step0,
                              float* epoch_loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    const int Bp = padded(batch);
    Carver cv(ws, ws_bytes);
    TrainWs w = carve_train<N>(cv, Bp);
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
            k_gather<N><<<ceil_div(Bq, 256), 256, 0, stream>>>(X, y, n, start, a, b, nv, Bq, w.Xb, w.XT, w.yb);
            if (batch_grad<N>(m, w, w.grad, nv, Bq, 1.f / (float)nv / (float)nb, epoch_loss + ep, stream) !=
                cudaSuccess)
                return BSPL_ECUDA;
            const int64_t k = (int64_t)ep * nb + bi;
            const float lr_k = lr * (1.f - 0.9f * (float)k / (float)total);
            if (launch_adam<N>(m, w.grad, adam_m, adam_v, ++step, lr_k, 0.9f, 0.999f, 1e-8f, stream) != cudaSuccess)
                return BSPL_ECUDA;
        }
    }
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_mlp_train(const bspl_mlp* m, float* adam_m, float* adam_v, int64_t n, const float* X,
                           const float* y, int32_t epochs, int32_t batch, float lr, uint64_t seed, int32_t step0,
                           float* epoch_loss, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!mlp_ok(m) || !adam_m || !adam_v || n < 1 || n > 0x7fffffffLL || !X || !y || epochs < 1 || batch < 1 ||
        batch > BSPL_MLP_MAX_BATCH || !epoch_loss || step0 < 0)
        return BSPL_EINVAL;
    if (!ws || ws_misaligned(ws) || ws_bytes < train_ws_bytes(m->kind, batch)) return BSPL_EINVAL;
    if (m->kind == BSPL_MLP_SURFACE)
        return train_impl<SurfNet>(m, adam_m, adam_v, n, X, y, epochs, batch, lr, seed, step0, epoch_loss, ws,
                                   ws_bytes, stream);
    return train_impl<CurveNet>(m, adam_m, adam_v, n, X, y, epochs, batch, lr, seed, step0, epoch_loss, ws, ws_bytes,
                                stream);
}

}  // extern "C"
