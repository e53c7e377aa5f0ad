// FMA-chain throughput microbenchmark (the ALU roofline denominators).
#include <cuda_runtime.h>

#include "../../include/bspl_measure.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma(int iters, T seed, T* sink)
{
    // 8 independent chains per thread keep every FMA pipe busy
    T a0 = seed + threadIdx.x, a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
    T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
    const T m = T(0.999999), c = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a0 = fma(a0, m, c);
            a1 = fma(a1, m, c);
            a2 = fma(a2, m, c);
            a3 = fma(a3, m, c);
            a4 = fma(a4, m, c);
            a5 = fma(a5, m, c);
            a6 = fma(a6, m, c);
            a7 = fma(a7, m, c);
        }
    }
    T r = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (r == T(-12345.678)) *sink = r;  // never true; keeps the chains live
}

template <class T>
int run(int iters, int reps, double* flops, void* sink, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 3;
    double best = 0.0;
    k_fma<T><<<blocks, threads, 0, s>>>(iters, T(0.5), (T*)sink);  // warm-up
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        k_fma<T><<<blocks, threads, 0, s>>>(iters, T(0.5), (T*)sink);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 3;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        double f = 2.0 * 64.0 * (double)iters * blocks * threads / (ms * 1e-3);
        if (f > best) best = f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops = best;
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace

extern "C" int bspl_measure_fma_peak(int fp64, int iters, int reps, double* flops, void* sink, cudaStream_t stream)
{
    if (!flops || !sink || iters <= 0 || reps <= 0) return 1;
    return fp64 ? run<double>(iters, reps, flops, sink, stream) : run<float>(iters, reps, flops, sink, stream);
}
