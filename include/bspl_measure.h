/*
 * bspl_measure.h -- measurement helper exported by libbspl (the paper has no
 * counterpart): the FP32 / FP64 FMA throughput of the GPU, used as the ALU
 * roofline denominator of the projection kernels.
 */
#ifndef BSPL_MEASURE_H
#define BSPL_MEASURE_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a grid of independent fused multiply-add chains (fp64 != 0: FP64,
 * else FP32) of `iters` steps per thread on `stream`, `reps` times, and
 * writes the best sustained rate in FLOP/s (2 per FMA) to *flops.  sink is a
 * device buffer of at least 4 bytes (receives a value that keeps the chains
 * alive).  Returns 0, or 3 when a CUDA call fails.  Allocates nothing. */
int bspl_measure_fma_peak(int fp64, int iters, int reps, double* flops, void* sink, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif
