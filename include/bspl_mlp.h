/*
 * bspl_mlp.h -- learned Newton seeds for the curve and surface queries of
 * libbspl.
 *
 * The paper has no learned component.  Its curve search stage (Sec. 4.2.3-
 * 4.4) finds, per query and segment, a start for the final Newton steps on
 * D(t) = |C(t) - q|^2 (Eqs. Dt, Et, E't); the grid search of
 * bspl_project_curves plays that role.  With opt->prec = BSPL_LEARNED_MIXED
 * and opt->mlp pointing to a bspl_mlp, a small network gives that start
 * instead, for every (query, segment) pair whose E = (C - q).C' has exactly
 * one root in (0, 1) with E(0) < 0 < E(1) (certified by the sign pattern of
 * E's Bernstein coefficients, Sec. 4.3 T matrix); every other pair keeps a
 * rule without a seed (an end of the segment, or the certified isolation of
 * E's roots).  FP32 Newton from the seed, two FP64 Newton steps, and the
 * FP64 safeguarded iteration as the fallback give the same results as the
 * other precisions (|d - d_oracle| <= 1e-9 x diag in the tests).
 *
 * Network: 15 inputs (+1 zero) -> 128 -> 128 -> 128 -> 1, GELU (tanh form)
 * after each hidden layer, logistic sigmoid on the output (t in (0, 1)).
 * Weights BF16, accumulation FP32 (tensor cores, tcgen05), activations
 * rounded to BF16 between layers.  Inputs, in the frame of the segment's
 * control-point box (centre c, scale s = 1 / longest side, no rotation):
 * (P_i - c) s for the four Bezier control points, then the query
 * v = (q - c) s with its part across the chord P0 -> P3 shortened to length
 * min(1, |part|) (the part along the chord is kept), then 0.
 *
 * Training (hand-written kernels, no library GEMM): mean squared error of t
 * against the FP64 minimiser t* of the pair, gradients by backpropagation
 * with BF16 operands and FP32 accumulation, Adam with bias correction on
 * FP32 master weights.
 *
 * Conventions as in bspl.h: device pointers owned by the caller, calls
 * asynchronous on the given stream, BSPL_EINVAL before any launch for bad
 * arguments, BSPL_ECUDA for launch failures.
 */
#ifndef BSPL_MLP_H
#define BSPL_MLP_H

#include "bspl.h"

#ifdef __cplusplus
extern "C" {
#endif

#define BSPL_MLP_IN 16
#define BSPL_MLP_HIDDEN 128
/* FP32 master parameter vector: offsets of each tensor (row-major [out][in]) */
#define BSPL_MLP_OFF_W1 0      /* [128][16] */
#define BSPL_MLP_OFF_B1 2048   /* [128] */
#define BSPL_MLP_OFF_W2 2176   /* [128][128] */
#define BSPL_MLP_OFF_B2 18560  /* [128] */
#define BSPL_MLP_OFF_W3 18688  /* [128][128] */
#define BSPL_MLP_OFF_B3 35072  /* [128] */
#define BSPL_MLP_OFF_W4 35200  /* [128] */
#define BSPL_MLP_OFF_B4 35328  /* [1], then 3 zeros */
#define BSPL_MLP_NPARAM 35332
/* BF16 copy read by the kernels: W1, W2, W3, W2^T, W3^T, w4 */
#define BSPL_MLP_NBF16 (2048 + 4 * 16384 + 128)
#define BSPL_MLP_MAX_BATCH 65536

/* The surface seed network (kind BSPL_MLP_SURFACE): 51 inputs (+13 zeros)
 * -> 128 -> 128 -> 128 -> 2, same activations; outputs (u, v) in (0, 1)^2,
 * the Newton start on a bicubic patch.  Inputs, in the frame of the patch's
 * control-net box (centre c, scale s = 1 / longest side): (P_ij - c) s for
 * the 16 Bezier control points (i along u, then j, then xyz), then the query
 * v = (q - c) s with its part along the normal of the frame e1 = P30 - P00,
 * e2 = (P03 - P00) without its e1 part, clamped to [-1, 1] (the tangential
 * parts are kept), then 13 zeros. */
#define BSPL_SMLP_IN 64
#define BSPL_SMLP_OUT 2
#define BSPL_SMLP_OFF_W1 0      /* [128][64] */
#define BSPL_SMLP_OFF_B1 8192   /* [128] */
#define BSPL_SMLP_OFF_W2 8320   /* [128][128] */
#define BSPL_SMLP_OFF_B2 24704  /* [128] */
#define BSPL_SMLP_OFF_W3 24832  /* [128][128] */
#define BSPL_SMLP_OFF_B3 41216  /* [128] */
#define BSPL_SMLP_OFF_W4 41344  /* [2][128] */
#define BSPL_SMLP_OFF_B4 41600  /* [2], then 2 zeros */
#define BSPL_SMLP_NPARAM 41604
#define BSPL_SMLP_NBF16 (8192 + 4 * 16384 + 256)

#define BSPL_MLP_CURVE 0   /* 16 -> 1 (t on a cubic segment) */
#define BSPL_MLP_SURFACE 1 /* 64 -> 2 ((u, v) on a bicubic patch) */

typedef struct {
    float* params;   /* device [BSPL_MLP_NPARAM] (curve) / [BSPL_SMLP_NPARAM]
                        (surface), FP32 master weights                         */
    uint16_t* wbf16; /* device [BSPL_MLP_NBF16] / [BSPL_SMLP_NBF16], BF16 copy
                        (round to nearest even), rewritten by bspl_mlp_sync and
                        bspl_mlp_adam                                          */
    int32_t kind;    /* BSPL_MLP_CURVE (0) or BSPL_MLP_SURFACE (1)             */
} bspl_mlp;

/* Every wait of the tensor-core kernels is bounded (1 s); a wait that gives
 * up sets a device flag and the kernel returns without its result.  This
 * call synchronises the stream, returns BSPL_ETIMEOUT (and clears the flag)
 * if any wait gave up since the last check, else BSPL_OK. */
bspl_status bspl_mlp_check(cudaStream_t stream);

/* Rewrites m->wbf16 from m->params. */
bspl_status bspl_mlp_sync(const bspl_mlp* m, cudaStream_t stream);

/* Fused inference on given inputs: X [n][in] FP32 -> t [n][out] (in, out =
 * 16, 1 for the curve network, 64, 2 for the surface network).  One kernel:
 * all four layers per tile of 128 rows, weights resident in shared memory,
 * accumulators in tensor memory. */
bspl_status bspl_mlp_forward(const bspl_mlp* m, int64_t n, const float* X, float* t, cudaStream_t stream);

/* Inputs of the (query, segment) pairs: pair_q [n] indexes q_xyz [.][3],
 * pair_seg [n] indexes the decomposition's segments -> X [n][16].
 * Out-of-range indices give a row of NaN. */
bspl_status bspl_mlp_features(const bspl_segments* segs, int64_t n, const int32_t* pair_q,
                              const int32_t* pair_seg, const double* q_xyz, float* X, cudaStream_t stream);

/* Training labels: t_star [n] = the minimiser of |C(u) - q|^2 over u in
 * [0, 1] on the pair's segment, FP64 (certified isolation of the roots of E
 * by Bernstein sign variations, bracketed Newton to 1e-15; ties -> the
 * smaller u), rounded to FP32.  Out-of-range indices give NaN. */
bspl_status bspl_mlp_labels(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_seg,
                            const double* q_xyz, float* t_star, cudaStream_t stream);

/* The (query, segment) pairs that the learned path seeds with the network
 * for the given queries (culling as in bspl_project_curves): at most cap
 * pairs are written to pair_q/pair_seg.  n_pairs (device, 2 values)
 * receives the number written and the number found (may exceed cap; pairs
 * are reserved in groups, so fewer than cap may be written when they do).
 * A candidate is filtered against its query's upper bound as it stands when
 * its warp classifies the buffered candidates, so the set can differ
 * slightly between calls (every set contains each query's minimiser).
 * Workspace: bspl_workspace_bytes(BSPL_OP_QUERY_CURVES_LEARNED, n, 0, 0, n_q). */
bspl_status bspl_mlp_collect_pairs(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                   const double* q_xyz, int64_t cap, int32_t* pair_q, int32_t* pair_seg,
                                   int64_t* n_pairs, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Loss and gradient for one batch (1 <= n <= BSPL_MLP_MAX_BATCH), X [n][in],
 * y [n][out]: loss (device scalar) = mean over rows and outputs of
 * (t - y)^2, grad [nparam] overwritten.
 * Workspace: bspl_workspace_bytes(BSPL_OP_MLP_TRAIN (curve) or
 * BSPL_OP_SMLP_TRAIN (surface), 0, 0, 0, n). */
bspl_status bspl_mlp_loss_grad(const bspl_mlp* m, int64_t n, const float* X, const float* y, float* grad,
                               float* loss, void* ws, size_t ws_bytes, cudaStream_t stream);

/* One Adam step (step counts from 1) on m->params, then m->wbf16 refreshed;
 * adam_m, adam_v [nparam] are the moment estimates (start at 0). */
bspl_status bspl_mlp_adam(const bspl_mlp* m, const float* grad, float* adam_m, float* adam_v, int32_t step,
                          float lr, float beta1, float beta2, float eps, cudaStream_t stream);

/* Whole training run on the stream: epochs x ceil(n / batch) Adam steps over
 * X [n][in], y [n][out]; each epoch visits the rows in the order
 * (a i + b) mod n with a, b drawn from seed (a coprime to n); the learning
 * rate falls linearly from lr to lr / 10; step numbering continues from
 * *step0 (0 for a fresh start).  epoch_loss [epochs] (device) receives the
 * mean batch loss of each epoch.
 * Workspace: bspl_workspace_bytes(BSPL_OP_MLP_TRAIN / BSPL_OP_SMLP_TRAIN, 0, 0,
 * 0, batch). */
bspl_status bspl_mlp_train(const bspl_mlp* m, float* adam_m, float* adam_v, int64_t n, const float* X,
                           const float* y, int32_t epochs, int32_t batch, float lr, uint64_t seed, int32_t step0,
                           float* epoch_loss, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Surface seed network: inputs of (query, patch) pairs -- pair_q [n] indexes
 * q_xyz [.][3], pair_patch [n] the decomposition's patches -> X [n][64]
 * (definition above; the control points come from the patch's FP32 power
 * coefficients, q - P00 is formed in FP64).  Out-of-range indices give NaN. */
bspl_status bspl_smlp_features(const bspl_segments* segs, int64_t n, const int32_t* pair_q,
                               const int32_t* pair_patch, const double* q_xyz, float* X, cudaStream_t stream);

/* Training labels of the surface network: uv [n][2] = the minimiser of
 * |S(u,v) - q|^2 over the pair's bicubic patch, (u, v) in [0,1]^2: a 17 x 17
 * FP32 sample grid in the frame of q, then FP64 projected Newton from its two
 * best samples (ties -> smaller u, then v), rounded to FP32.  Out-of-range
 * indices give NaN. */
bspl_status bspl_smlp_labels(const bspl_segments* segs, int64_t n, const int32_t* pair_q, const int32_t* pair_patch,
                             const double* q_xyz, float* uv, cudaStream_t stream);

/* The (query, patch) pairs the learned surface path seeds with the network
 * for the given queries (the surface culling of bspl_project_surfaces, at
 * most 64 pairs per query; a query with more is left to the sample grid and
 * contributes none): at most cap pairs are written to pair_q (the query's
 * index) / pair_patch; n_pairs (device, 2 values) receives the number
 * written and the number found.
 * Workspace: bspl_workspace_bytes(BSPL_OP_QUERY_SURFACES_LEARNED, n, 0, 0, n_q). */
bspl_status bspl_smlp_collect_pairs(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf,
                                    const double* q_xyz, int64_t cap, int32_t* pair_q, int32_t* pair_patch,
                                    int64_t* n_pairs, void* ws, size_t ws_bytes, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* BSPL_MLP_H */
