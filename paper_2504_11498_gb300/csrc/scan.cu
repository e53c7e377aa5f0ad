// Exclusive prefix sum of int64 counts (segment offsets, query buckets).
// Three-phase: per-block scan writing block totals, recursive scan of the
// totals, then a uniform add.  2048 elements per block of 512 threads.
#include "bspl_internal.cuh"

namespace bspl {

namespace {
constexpr int kThreads = 512;
constexpr int kPer = 4;
constexpr int kTile = kThreads * kPer;

__global__ void block_scan(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                           int64_t* __restrict__ sums)
{
    __shared__ int64_t warp_tot[kThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPer;
    int64_t v[kPer];
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        acc += v[k];
    }
    // inclusive scan of per-thread totals within the warp
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < kThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t run = x - acc + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == kThreads - 1 && sums) sums[blockIdx.x] = run;
}

__global__ void add_block_offsets(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t add = sums[blockIdx.x];
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}
}  // namespace

size_t scan_tmp_elems(int64_t n)
{
    size_t total = 0;
    while (n > kTile) {
        n = (n + kTile - 1) / kTile;
        total += (size_t)n;
    }
    return total + 1;
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + kTile - 1) / kTile;
    if (nb == 1) {
        block_scan<<<1, kThreads, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int64_t* sums = tmp;
    block_scan<<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = exclusive_scan_i64(sums, sums, nb, tmp + nb, s);
    if (e != cudaSuccess) return e;
    add_block_offsets<<<(unsigned)nb, kThreads, 0, s>>>(out, n, sums);
    return cudaGetLastError();
}

}  // namespace bspl
