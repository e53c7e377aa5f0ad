// extern "C" entry points of libbspl (declared in include/bspl.h): argument
// checks and dispatch to the kernels.
#include "bspl_internal.cuh"

using namespace bspl;

namespace {
// Every entry point reports the failures of its own CUDA calls: a launch
// error left over from an earlier call (kept by the runtime until read) is
// read and dropped first.
inline void clear_stale_error() { (void)cudaGetLastError(); }
}  // namespace

extern "C" {

size_t bspl_workspace_bytes(int op, int64_t n_splines, int64_t n_cp_total, int64_t n_seg, int64_t n_q)
{
    (void)n_seg;
    if (n_splines < 0 || n_cp_total < 0 || n_q < 0) return 0;
    switch (op) {
    case BSPL_OP_DECOMPOSE_CURVES: return decompose_ws_bytes(0, n_splines, n_cp_total);
    case BSPL_OP_DECOMPOSE_SURFACES: return decompose_ws_bytes(1, n_splines, n_cp_total);
    case BSPL_OP_QUERY_CURVES:
    case BSPL_OP_QUERY_SURFACES: return query_ws_bytes(n_splines, n_q);
    case BSPL_OP_QUERY_CURVES_LEARNED: return learned_ws_bytes(n_splines, n_q);
    case BSPL_OP_MLP_TRAIN: return n_q >= 1 && n_q <= 65536 ? train_ws_bytes(0, n_q) : 0;
    case BSPL_OP_SMLP_TRAIN: return n_q >= 1 && n_q <= 65536 ? train_ws_bytes(1, n_q) : 0;
    case BSPL_OP_QUERY_SURFACES_LEARNED: return learned_surf_ws_bytes(n_splines, n_q);
    case BSPL_OP_REFINE_CURVES: return refine_ws_bytes(n_splines, n_cp_total, n_q);
    default: return 0;
    }
}

bspl_status bspl_decompose(int is_surface, const void* splines, double tol_rel, bspl_segments* out,
                           int64_t* n_seg_total, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    if (is_surface) return decompose_surfaces((const bspl_surfaces*)splines, tol_rel, out, n_seg_total, ws, ws_bytes,
                                              stream);
    return decompose_curves((const bspl_curves*)splines, tol_rel, out, n_seg_total, ws, ws_bytes, stream);
}

bspl_status bspl_project_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                                const bspl_options* opt, double* t, double* dist, uint8_t* status, void* ws,
                                size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    return query_curves(segs, n_q, q_curve, q_xyz, opt, 0, t, dist, status, ws, ws_bytes, stream);
}

bspl_status bspl_invert_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                               const bspl_options* opt, double* t, double* dist, uint8_t* status, void* ws,
                               size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    return query_curves(segs, n_q, q_curve, q_xyz, opt, 1, t, dist, status, ws, ws_bytes, stream);
}

bspl_status bspl_project_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf, const double* q_xyz,
                                  const bspl_options* opt, double* uv, double* dist, uint8_t* status, void* ws,
                                  size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    return query_surfaces(segs, n_q, q_surf, q_xyz, opt, 0, uv, dist, status, ws, ws_bytes, stream);
}

bspl_status bspl_invert_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf, const double* q_xyz,
                                 const bspl_options* opt, double* uv, double* dist, uint8_t* status, void* ws,
                                 size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    return query_surfaces(segs, n_q, q_surf, q_xyz, opt, 1, uv, dist, status, ws, ws_bytes, stream);
}

bspl_status bspl_eval_curves(const bspl_curves* curves, int64_t n_q, const int32_t* q_curve, const double* t,
                             double* xyz, cudaStream_t stream)
{
    clear_stale_error();
    return eval_curves(curves, n_q, q_curve, t, xyz, stream);
}

bspl_status bspl_eval_surfaces(const bspl_surfaces* surfaces, int64_t n_q, const int32_t* q_surf, const double* uv,
                               double* xyz, cudaStream_t stream)
{
    clear_stale_error();
    return eval_surfaces(surfaces, n_q, q_surf, uv, xyz, stream);
}

bspl_status bspl_refine_curves(const bspl_curves* curves, const double* diag, int invert, int64_t n_q,
                               const int32_t* q_curve, const double* q_xyz, int32_t max_iter, double* t,
                               double* dist, uint8_t* status, uint64_t* evals, void* ws, size_t ws_bytes,
                               cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    clear_stale_error();
    return refine_curves(curves, diag, invert, n_q, q_curve, q_xyz, max_iter, t, dist, status, evals, ws, ws_bytes,
                         stream);
}

const char* bspl_status_string(bspl_status s)
{
    switch (s) {
    case BSPL_OK: return "BSPL_OK";
    case BSPL_EINVAL: return "BSPL_EINVAL";
    case BSPL_ENOSPACE: return "BSPL_ENOSPACE";
    case BSPL_ECUDA: return "BSPL_ECUDA";
    case BSPL_ENOTCONV: return "BSPL_ENOTCONV";
    case BSPL_ETIMEOUT: return "BSPL_ETIMEOUT";
    default: return "BSPL_UNKNOWN";
    }
}

}  // extern "C"
