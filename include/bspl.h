/*
 * bspl.h -- C ABI of the GB300 (sm_103a) library for batched point projection
 * and inversion on B-spline curves (non-rational and rational) and
 * non-rational B-spline surfaces, after their decomposition into cubic
 * Bezier segments / bicubic Bezier patches.
 *
 * Method: Wu & Zou, "Matrix representation and GPU-optimized parallel
 * B-spline computing" (arXiv 2504.11498).
 *   - problem statement: Sec. 3, Eqs. projection, projections, inversion;
 *   - decomposition: Sec. 4.2.1 (Eq. decomfinal) and Sec. 4.2.2 (G1-continuous
 *     degree reduction, Eqs. G1-condition, epsl, differentiatedelta0/1;
 *     error-controlled subdivision, Eq. subLandR);
 *   - squared distance and its derivatives: Sec. 4.2.3, Eqs. Dt, Et, E't;
 *   - per-query minimum and reparameterisation: Sec. 4.4.2.
 *
 * Conventions for every entry point:
 *   - all array pointers are DEVICE pointers owned by the caller unless stated
 *     otherwise; the library never allocates or frees device memory;
 *   - every call is asynchronous on the given stream, except bspl_decompose,
 *     which synchronises that stream (after validating the splines, after
 *     counting the segments, and around computing spline_rank);
 *   - a workspace (ws) must start on a 256-byte boundary, as cudaMalloc
 *     returns (the library carves it at 256-byte offsets);
 *   - argument errors that the host can see (NULL pointers, negative sizes,
 *     workspace too small or misaligned) return BSPL_EINVAL before anything
 *     is launched;
 *     per-query data problems (spline index out of range, non-finite point)
 *     set BSPL_Q_INVALID in that query's status byte; nothing traps;
 *   - CUDA launch failures return BSPL_ECUDA.
 */
#ifndef BSPL_H
#define BSPL_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BSPL_OK = 0,
    BSPL_EINVAL = 1,   /* invalid argument or spline data                       */
    BSPL_ENOSPACE = 2, /* capacity too small (counts were still written)        */
    BSPL_ECUDA = 3,    /* a CUDA call failed                                    */
    BSPL_ENOTCONV = 4, /* subdivision hit its depth cap (40) somewhere          */
    BSPL_ETIMEOUT = 5  /* a bounded device wait gave up (bspl_mlp_check)        */
} bspl_status;

typedef enum {
    BSPL_FP64 = 0,          /* cull, seed and Newton all in FP64                  */
    BSPL_MIXED = 1,         /* FP32 cull/seed/early Newton + 2 FP64 Newton steps  */
    BSPL_LEARNED_MIXED = 2, /* as MIXED with the MLP seed in place of the grid
                               (bspl_mlp.h; surfaces: the surface network)      */
    BSPL_CLIP_MIXED = 3     /* curves: the learned path's culling and
                               certification with the paper's search (Secs.
                               4.2.3-4.4: monotone split by the closed-form
                               roots of E', elimination by Properties 1-2,
                               Bezier clipping to 1e-6 of each piece) in place
                               of the network and of the FP32 root isolation,
                               then the FP32 and FP64 Newton steps; surfaces:
                               EINVAL                                          */
} bspl_precision;

/* per-query status bits */
#define BSPL_Q_CONVERGED 1u  /* the final Newton step met its tolerance          */
#define BSPL_Q_FALLBACK 2u   /* mixed/learned result needed the FP64 fallback
                                (safeguarded iteration, or the certified FP64
                                isolation of the segment's minima)              */
#define BSPL_Q_AT_END 4u     /* minimiser at an end of the parameter domain      */
#define BSPL_Q_NONCONV 8u    /* Newton cap reached without convergence           */
#define BSPL_Q_OFF_CURVE 16u /* inversion: distance above 1e-9 x diagonal        */
#define BSPL_Q_INVALID 32u   /* spline index out of range or non-finite point    */

/* Curves in CSR form (Sec. 3): curve c has degree p = degree[c] (1..63;
 * the paper's method stops at 31; see bspl_decompose for degrees above 7),
 * control points cps[cp_off[c] .. cp_off[c+1]) (xyz, FP64, [ncp][3]) and
 * knots knots[knot_off[c] .. knot_off[c+1]) with ncp + p + 1 entries,
 * non-decreasing and finite.  The parameter domain is [t_p, t_{ncp}].
 *
 * weights: NULL for non-rational curves (the paper's setting), else one
 * finite positive weight per control point (weights[cp_off[c] + i] belongs
 * to cps[cp_off[c] + i]) and the curves are rational (NURBS):
 *   C(t) = sum_i N_{i,p}(t) w_i P_i / sum_i N_{i,p}(t) w_i.
 * The paper names rational splines as outside its method; here the
 * decomposition, the evaluation and the refinement take them (see
 * bspl_decompose and bspl_refine_curves), and the query calls search the
 * cubic Beziers the decomposition returns exactly as for any other curve.
 * A curve whose weights are all equal is the non-rational curve and is
 * treated as one. */
typedef struct {
    int64_t n;
    const int32_t* degree;
    const int64_t* knot_off;
    const double* knots;
    const int64_t* cp_off;
    const double* cps;
    const double* weights;
} bspl_curves;

/* Tensor-product surfaces in CSR form: surface s has degrees deg_u[s],
 * deg_v[s] (1..7; the span-pair nets the query kernels keep are 8 x 8;
 * other degrees -> BSPL_EINVAL), an n_u[s] x n_v[s] control net stored row-major
 * [n_u][n_v][3] (first index along u) at cps[3*cp_off[s]...], and knot
 * vectors knots_u[knot_u_off[s]..], knots_v[knot_v_off[s]..] of lengths
 * n_u+deg_u+1 and n_v+deg_v+1. */
typedef struct {
    int64_t n;
    const int32_t* deg_u;
    const int32_t* deg_v;
    const int32_t* n_u;
    const int32_t* n_v;
    const int64_t* knot_u_off;
    const double* knots_u;
    const int64_t* knot_v_off;
    const double* knots_v;
    const int64_t* cp_off;
    const double* cps;
} bspl_surfaces;

/* widths (in elements) of the per-segment and per-group records */
#define BSPL_GROUP 32        /* consecutive segments/patches per culling group */
#define BSPL_CREC64 18       /* curve FP64: lo[3] hi[3] a0[3] a1[3] a2[3] a3[3] (power basis in u) */
#define BSPL_CREC32 24       /* curve FP32: same layout (box rounded outward), then a0 - (float)a0 [3] and 3 pad */
#define BSPL_SREC64 54       /* patch FP64: lo[3] hi[3] a[4][4][3] (power basis in u,v) */
#define BSPL_SREC32 72       /* patch FP32: same layout, then [54] pu, [55] pv (span-pair
                                degrees), [56..60] bounds of the ORIGINAL piece's
                                |S_s|, |S_t|, |S_ss|, |S_st|, |S_tt| over the patch in
                                its own parameters (s, t) in [0,1]^2, [61] edge flags
                                (bit 0: s=0, 1: s=1, 2: t=0, 3: t=1 set where the
                                surface is C1 across that edge), [62..65] bounds of
                                |S_sss|, |S_sst|, |S_stt|, |S_ttt|, [66..71] the sums
                                over the non-constant terms s^i t^j of patch_net32 of
                                |coefficient| x 1, i, j, i(i-1), ij, j(j-1) (summed over
                                xyz, rounded up): the norms that bound the rounding of
                                the FP32 search's Horner evaluation */
#define BSPL_GREC64 12       /* group FP64: lo[3] hi[3] ref[3] pad[3] */
#define BSPL_GREC32 12       /* group FP32: same, box rounded outward */

/* Decomposition output and query tables (all caller-owned device memory).
 *   seg_off [n+1]        segments of spline i are [seg_off[i], seg_off[i+1])
 *   ctrl    [cap][4][3]  cubic Bezier control points (curves)
 *           [cap][4][4][3] bicubic net, first index along u (surfaces)
 *   prange  [cap][2]     (t0, t1) of each segment in the original parameter
 *           [cap][4]     (u0, u1, v0, v1) of each patch
 *   diag    [n]          diagonal of each spline's control-point box (NaN
 *                        for a spline that failed validation)
 *   rec64/rec32          per-segment search records (BSPL_*REC* above); rec32
 *                        and grp32 must be 16-byte aligned (the query kernels
 *                        stage them into shared memory by bulk copies)
 *   grp_off [n+1], grp64/grp32: culling groups of BSPL_GROUP consecutive
 *                        segments (box of the group + a point on it);
 *                        grp_capacity >= n + capacity / BSPL_GROUP + 1 always suffices
 * Surfaces additionally:
 *   patch_span [cap] int64  span-pair slot of each patch
 *   patch_box  [cap][4]     the patch's (u0,u1,v0,v1) inside its span pair, in [0,1]
 *   span_net   [n_cp_total][BSPL_SPAN_NET]  power-basis coefficients of the
 *                        ORIGINAL span-pair patch (degree <= 7 per direction in
 *                        the query path), indexed by slot, used for the final
 *                        FP64 Newton steps on the original surface;
 *   span_net32 [n_cp_total][BSPL_SPAN_NET]  the same in FP32 (mixed precision);
 *   patch_net32 [cap][BSPL_SPAN_NET]  the ORIGINAL piece over each patch's own
 *                        parameter box, in the patch's power basis (s, t in
 *                        [0,1]^2), FP32, same layout as span_net; its constant
 *                        term is the patch corner, whose FP64 value is
 *                        rec64[6..8].  Coefficients of the patch's size keep
 *                        the FP32 search accurate on small patches.
 */
#define BSPL_SPAN_NET (8 * 8 * 3)
typedef struct {
    int32_t is_surface;
    int64_t n;
    int64_t capacity;
    int64_t grp_capacity;
    int64_t* seg_off;
    double* ctrl;
    double* prange;
    double* diag;
    double* rec64;
    float* rec32;
    int64_t* grp_off;
    double* grp64;
    float* grp32;
    int64_t* patch_span;
    double* patch_box;
    double* span_net;
    float* span_net32;
    int64_t n_cp_total;  /* in: cp_off[n] of the decomposed set (sizes the slot arrays) */
    double tol_rel;      /* out: tolerance the tables were built with */
    float* patch_net32;  /* surfaces: [capacity][BSPL_SPAN_NET], see above */
    int32_t* spline_rank;/* optional [n]: rank of each spline by descending piece
                            count (ties by index), written by the filling pass;
                            the query calls then group queries heaviest spline
                            first, which their work-stealing launch hands out
                            first.  NULL: queries grouped by spline index. */
} bspl_segments;

/* Query options.  Zero fields take the defaults given. */
typedef struct {
    int32_t prec;        /* bspl_precision (default BSPL_FP64)                      */
    int32_t samples;     /* grid samples per segment/patch: 8, 16 or 32 (curves, default
                            16; 8 is coarse and may miss close minima), 16 or 32
                            (surfaces, 4x4 or 8x4, default 32)                   */
    int32_t newton_max;  /* FP64 Newton cap, plain path and fallback (default 30)   */
    int32_t fp32_steps;  /* FP32 Newton steps before the FP64 finish (default 4 for
                            curves, 8 per stage for surfaces)               */
    int32_t sort_queries;/* 1: group queries by spline first (default 1)            */
    int32_t occupancy;   /* curve kernel register/occupancy variant: 0 compiler
                            choice, 1 >= 4 blocks/SM, 2 >= 6 blocks/SM (samples
                            16 and 32); learned path: 0 compiler choice, 1 / 2
                            culling kernel fitted to 6 / 8 blocks/SM; picked
                            by the autotuner                                */
    int32_t pairs_per_query; /* learned path: candidate-pair buffer per query,
                            1..24 (default 24); queries whose pairs do not fit
                            are answered by the grid kernel instead         */
    const void* mlp;     /* BSPL_LEARNED_MIXED: const bspl_mlp* (bspl_mlp.h) giving
                            the Newton seed; NULL -> the seed is u = 1/2 (the
                            learned path without its network)               */
    uint64_t* counters;  /* optional device array [BSPL_NCOUNTERS], accumulated     */
    const void* stage_events; /* optional host array of BSPL_NSTAGE_EVENTS cudaEvent_t
                            (created by the caller): the learned path records
                            them on the stream at its stage boundaries (start,
                            sort, cull, classify, seed, FP32, FP64, select,
                            leftovers); profiling only                    */
    int32_t cert_depth;  /* surfaces: refinement levels of the certification
                            search on the original surface (default 2, at most
                            4); negative: no certification (grid-seeded search
                            only, for timing comparisons)                 */
} bspl_options;
#define BSPL_NSTAGE_EVENTS 9

/* device counters accumulated by the query calls when opt->counters != NULL */
#define BSPL_CNT_QUERIES 0
#define BSPL_CNT_SEG_TESTED 1  /* segment boxes tested */
#define BSPL_CNT_GRP_TESTED 2  /* group boxes tested */
#define BSPL_CNT_CANDIDATES 3  /* segments that reached the seed stage */
#define BSPL_CNT_NEWTON 4      /* Newton candidates (basins) refined */
#define BSPL_CNT_FALLBACK 5    /* queries that needed the FP64 fallback */
#define BSPL_CNT_NONCONV 6
#define BSPL_CNT_NEWTON32_ITERS 7 /* FP32 Newton iterations */
#define BSPL_CNT_NEWTON64_ITERS 8 /* FP64 Newton iterations */
#define BSPL_CNT_ISO_PAIRS 9   /* learned path: pairs sent to certified root isolation */
#define BSPL_CNT_CERT_CELLS 10 /* surfaces: cells evaluated by the certification search */
#define BSPL_CNT_CERT_LEAVES 11 /* surfaces: certification cells handed to Newton */
#define BSPL_CNT_CERT_OVERFLOW 12 /* surfaces: cells sent to Newton early (stack full) */
#define BSPL_CNT_CLASSIFIED 13 /* learned path: pairs classified by the Bernstein signs of E */
#define BSPL_NCOUNTERS 14

/* workspace sizes: op is one of */
#define BSPL_OP_DECOMPOSE_CURVES 1
#define BSPL_OP_DECOMPOSE_SURFACES 2
#define BSPL_OP_QUERY_CURVES 3
#define BSPL_OP_QUERY_SURFACES 4
#define BSPL_OP_QUERY_CURVES_LEARNED 5 /* curve queries with opt->prec = BSPL_LEARNED_MIXED */
#define BSPL_OP_MLP_TRAIN 6            /* bspl_mlp_loss_grad / bspl_mlp_train, n_q = batch */
#define BSPL_OP_SMLP_TRAIN 7           /* the same for the surface seed network */
#define BSPL_OP_QUERY_SURFACES_LEARNED 8 /* surface queries with opt->prec = BSPL_LEARNED_MIXED */
#define BSPL_OP_REFINE_CURVES 9          /* bspl_refine_curves grouping its queries by curve */

/* Bytes of device workspace a call of kind `op` needs.  n_splines = n,
 * n_cp_total = total control points (cp_off[n]), n_seg = segments of the
 * decomposition, n_q = queries. */
size_t bspl_workspace_bytes(int op, int64_t n_splines, int64_t n_cp_total, int64_t n_seg, int64_t n_q);

/* Decomposes every spline into cubic Bezier segments (is_surface = 0,
 * splines -> bspl_curves) or bicubic patches (is_surface = 1, splines ->
 * bspl_surfaces), Sec. 4.2:
 *   each non-empty knot span (span pair) is converted to its Bezier piece by
 *   the span-wise matrix route Q = B_p^{-1} M A P (Eq. decomfinal, formed in
 *   the local parameter); degree 1-2 pieces are elevated exactly, degree 3
 *   kept, higher degrees reduced by the G1-continuous L2-optimal rule; a
 *   reduced piece whose certified deviation bound (control points of the
 *   difference after elevation) exceeds tol_rel x diag is split at the
 *   midpoint of its parameter interval and both halves are reduced again
 *   from the original piece (depth cap 40 and at most 65536 pieces per span
 *   or span pair; reaching either accepts the piece and -> BSPL_ENOTCONV).
 * Degrees 8..63: the power-basis coefficients of the matrix route grow like
 * C(p, p/2) and take as many digits (measured against knot insertion:
 * 6e-14 of the control points' size at degree 7, 2e-10 at 15, 1e-2 at 31,
 * the paper's own limit), so above degree 7 each span's Bezier points are
 * the blossom values at the span's end knots instead (de Boor's algorithm:
 * convex combinations of the span's control points), then reduced, bounded
 * and subdivided as above.
 * Rational curves (bspl_curves.weights, weights not all equal): the matrix
 * route is applied to the homogeneous control points (w_i P_i, w_i), which
 * gives each span's rational Bezier piece as homogeneous points (W_j Q_j,
 * W_j); a piece (or a half of one, by de Casteljau halving of the
 * homogeneous points) is replaced by the C1 Hermite cubic of its end points
 * and end derivatives, accepted when the certified bound
 * max_k |(A - W R)_k| / min_j W_j (Bernstein coefficients of A - W R at
 * degree p + 3, A and W the numerator and weight of the piece, R the
 * cubic) is at most tol_rel x diag, else split at the midpoint like a
 * reduced piece (same caps).
 * Two-phase use: with out->ctrl == NULL the call only counts: it writes
 * out->seg_off, out->diag and *n_seg_total and returns BSPL_OK.  Otherwise,
 * if *n_seg_total > out->capacity (or the group count exceeds
 * out->grp_capacity) it writes the counts and returns BSPL_ENOSPACE; else it
 * fills every array of *out.  out->n_cp_total must equal cp_off[n].
 * Invalid spline data (degree out of range, knot count
 * mismatch, decreasing or non-finite knots, non-finite control points, a
 * weight that is not finite and positive, empty domain) -> BSPL_EINVAL with
 * nothing written beyond seg_off/diag.
 * Workspace: bspl_workspace_bytes(BSPL_OP_DECOMPOSE_*, n, n_cp_total, 0, 0). */
bspl_status bspl_decompose(int is_surface, const void* splines, double tol_rel, bspl_segments* out,
                           int64_t* n_seg_total, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Projection of n_q points q_xyz [n_q][3] onto curves q_curve [n_q] (Eq.
 * projections): t [n_q] receives the minimising parameter in the curve's
 * original parameter (Sec. 4.4.2 reparameterisation), dist [n_q] the distance
 * to the decomposed curve, status [n_q] the BSPL_Q_* bits.  Search: group
 * queries by curve, cull segment groups and segments by box distance against
 * an upper bound from points on the curve, sample a grid on each surviving
 * segment, refine every sampled basin by safeguarded Newton on E = D'
 * (Eqs. Dt, Et, E't), keep the smallest distance (ties: smallest parameter).
 * opt->prec selects FP64 or FP32 search + 2 FP64 Newton steps; with
 * BSPL_LEARNED_MIXED every surviving (query, segment) pair is classified by
 * the signs of E's Bernstein coefficients (Sec. 4.3) instead of sampled, the
 * single-minimum pairs are seeded by the network (bspl_mlp.h), and pairs the
 * FP32 stage cannot settle are decided in FP64 (the certified isolation when
 * needed); at most 89,478,314 queries per call (the pair buffer is indexed
 * in 32 bits).
 * Workspace: bspl_workspace_bytes(BSPL_OP_QUERY_CURVES, n, n_cp_total, n_seg, n_q)
 * (BSPL_OP_QUERY_CURVES_LEARNED for the learned path). */
bspl_status bspl_project_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                const double* q_xyz, const bspl_options* opt, double* t, double* dist,
                                uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Inversion (Eq. inversion): the same search for points that lie on the
 * curve; additionally sets BSPL_Q_OFF_CURVE when dist > 1e-9 x diag. */
bspl_status bspl_invert_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                               const double* q_xyz, const bspl_options* opt, double* t, double* dist,
                               uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Surface projection: uv [n_q][2] receives the minimising (u, v) in the
 * surface's original parameters, dist the distance to the ORIGINAL surface
 * (the last two FP64 Newton steps run on the original span-pair patch).
 * Workspace: bspl_workspace_bytes(BSPL_OP_QUERY_SURFACES, ...). */
bspl_status bspl_project_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf,
                                  const double* q_xyz, const bspl_options* opt, double* uv, double* dist,
                                  uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Surface inversion; sets BSPL_Q_OFF_CURVE when dist > 1e-9 x diag. */
bspl_status bspl_invert_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf,
                                 const double* q_xyz, const bspl_options* opt, double* uv, double* dist,
                                 uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t stream);

/* Scratch-free projection (the paper has no counterpart).
 *
 * Same computation and results as bspl_project_curves, for callers that
 * cannot allocate device memory for a workspace: for example an application
 * that hands all GPU memory to its own pool up front, a plugin or callback
 * that is not allowed to call the CUDA allocator, or a latency-critical loop
 * where an allocation and its implicit synchronisation are not acceptable.
 * The caller still owns and passes the inputs and the outputs; the scratch
 * (the per-curve query buckets and the query order) lives in a fixed
 * BSPL_NOALLOC_SCRATCH_BYTES array inside the library, which every GPU that
 * loads the library keeps reserved until the process exits.
 *
 * Limits: n_q <= BSPL_NOALLOC_MAX_QUERIES and segs->n <= BSPL_NOALLOC_MAX_SPLINES.
 * With opt->prec = BSPL_LEARNED_MIXED the culling-candidate and pair buffers
 * (about 1.4 KB per query) share the array, which lowers the limit to about
 * 5,800 queries
 * (exactly: bspl_workspace_bytes(BSPL_OP_QUERY_CURVES_LEARNED, segs->n, 0, 0,
 * n_q) must not exceed BSPL_NOALLOC_SCRATCH_BYTES).  Larger calls return
 * BSPL_ENOSPACE before anything is launched.
 * The first call on a device looks up the array's device address for that
 * device (with that device current); make that first call before any stream
 * capture.  All calls share the one array: its contents are those of the
 * last call, each call clears what must start at zero, and calls that
 * overlap on the GPU (for example on two streams at once) race with each
 * other.  Nothing is allocated or freed. */
#define BSPL_NOALLOC_MAX_QUERIES (1 << 20)
#define BSPL_NOALLOC_MAX_SPLINES (1 << 18)
#define BSPL_NOALLOC_SCRATCH_BYTES (8u << 20)
bspl_status bspl_project_curves_noalloc(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                        const double* q_xyz, const bspl_options* opt, double* t, double* dist,
                                        uint8_t* status, cudaStream_t stream);

/* Evaluates the ORIGINAL curves at t [n_q] (Cox-de Boor, Sec. 3 Eq.
 * bsplinebasis; rational curves: the homogeneous sums divided by the
 * weight sum): xyz [n_q][3].  t outside the domain is clamped; an
 * out-of-range curve index yields NaN.  Used to place inversion queries. */
bspl_status bspl_eval_curves(const bspl_curves* curves, int64_t n_q, const int32_t* q_curve, const double* t,
                             double* xyz, cudaStream_t stream);

/* Evaluates the ORIGINAL surfaces at uv [n_q][2]: xyz [n_q][3]. */
bspl_status bspl_eval_surfaces(const bspl_surfaces* surfaces, int64_t n_q, const int32_t* q_surf,
                               const double* uv, double* xyz, cudaStream_t stream);

/* Refines curve projection / inversion results on the ORIGINAL curves (the
 * problem of Sec. 3, Eqs. projection and inversion, posed on C itself rather
 * than on the cubic approximant the query calls search): from t [n_q] (the
 * original parameter, as bspl_project_curves / bspl_invert_curves return
 * it), FP64 Newton on E = (C - q).C', E' = C'.C' + (C - q).C'' (Sec. 4.2.3,
 * Eqs. Et and E't) with C, C', C'' by the Cox-de Boor recursion on the
 * original knots and control points (rational curves: on the homogeneous
 * points, then C = A/W, C' = (A' - W'C)/W, C'' = (A'' - 2W'C' - W''C)/W, the
 * quotient rule: rational Newton); every step is clamped to the domain and
 * halved (at most 12 times) until the squared distance does not grow (a full
 * step that leaves the knot span of t is first replaced by the knot it
 * crossed, where a C0 joint may hold the minimum), until E is zero to its
 * FP64 rounding, the step falls below the resolution of t or the distance
 * stops decreasing.  At most max_iter steps (0: 16; at most 100).
 *   in/out  t [n_q], dist [n_q]: the refined parameter and |C(t) - q|, never
 *           larger than the distance at the starting t beyond the FP64
 *           rounding of the squared distance (a full Newton step whose
 *           change of it is within that rounding is taken and ends the
 *           iteration);
 *   in/out  status [n_q]: queries with BSPL_Q_INVALID are skipped; otherwise
 *           CONVERGED / NONCONV and AT_END are set from the refinement and,
 *           with invert != 0 and diag != NULL (the per-curve diagonals, e.g.
 *           bspl_segments.diag), OFF_CURVE from the refined distance.
 * The result is the local minimum of the original curve reached from the
 * approximant's answer: it is the global one unless the original curve has
 * another local minimum whose distance is within twice the decomposition
 * tolerance of it.  Degrees 1..63 (others are left unchanged).
 *   out     evals: optional device array [BSPL_REFINE_EVALS], accumulated:
 *           entry p counts the evaluations of C, C', C'' on curves of
 *           degree p, entry 32 + p those of C and C' alone (the trial points
 *           of the steps) (profiling; NULL: not counted).
 *   ws      optional device workspace of
 *           bspl_workspace_bytes(BSPL_OP_REFINE_CURVES, curves->n,
 *           cp_off[n], 0, n_q) bytes: the queries are then processed grouped
 *           by curve (a warp's queries share a curve's degree and knots), and
 *           the factors of each span's evaluation that depend on the knots
 *           alone (reciprocals of knot differences, for degrees up to 7) are
 *           computed once per span for the call instead of once per query;
 *           a smaller workspace (at least the n_cp_total = 0 size) groups the
 *           queries and keeps the factors of the curves that fit.  NULL: the
 *           caller's order, factors per query.  The results do not depend on
 *           either (same operations).
 * BSPL_EINVAL for NULL arrays with n_q > 0, n_q < 0, max_iter outside
 * 0..100, or a workspace given with ws_bytes below the n_cp_total = 0 size
 * above. */
bspl_status bspl_refine_curves(const bspl_curves* curves, const double* diag, int invert, int64_t n_q,
                               const int32_t* q_curve, const double* q_xyz, int32_t max_iter, double* t,
                               double* dist, uint8_t* status, uint64_t* evals, void* ws, size_t ws_bytes,
                               cudaStream_t stream);

#define BSPL_REFINE_EVALS 64

/* Human-readable name of a status code (static string). */
const char* bspl_status_string(bspl_status s);

#ifdef __cplusplus
}
#endif
#endif /* BSPL_H */
