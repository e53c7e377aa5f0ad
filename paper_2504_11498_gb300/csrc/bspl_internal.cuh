// Internal declarations shared by the CUDA translation units of libbspl.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bspl.h"

namespace bspl {

constexpr int kMaxCurveDegree = 31;
constexpr int kMaxSurfDegree = 7;
constexpr int kDepthCap = 40;
constexpr int64_t kLeafCap = 65536;  // leaves per span (pair) after which every node is accepted

// ---------------------------------------------------------------- workspace
// Carves caller workspace into aligned sub-buffers.
struct Carver {
    char* base;
    size_t used, cap;
    __host__ Carver(void* p, size_t n) : base((char*)p), used(0), cap(n) {}
    template <class T>
    __host__ T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        if (base == nullptr) return nullptr;
        return used <= cap ? (T*)(base + off) : nullptr;
    }
};

// exclusive scan of int64 values (in place allowed); tmp from the workspace
size_t scan_tmp_elems(int64_t n);
cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);

// decomposition entry points (decompose.cu)
bspl_status decompose_curves(const bspl_curves* c, double tol_rel, bspl_segments* out, int64_t* total,
                             void* ws, size_t ws_bytes, cudaStream_t s);
bspl_status decompose_surfaces(const bspl_surfaces* c, double tol_rel, bspl_segments* out, int64_t* total,
                               void* ws, size_t ws_bytes, cudaStream_t s);
size_t decompose_ws_bytes(int is_surface, int64_t n, int64_t n_cp_total);

// queries (query_curves.cu, query_surfaces.cu)
bspl_status query_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                         const bspl_options* opt, int invert, double* t, double* dist, uint8_t* status, void* ws,
                         size_t ws_bytes, cudaStream_t s);
bspl_status query_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf, const double* q_xyz,
                           const bspl_options* opt, int invert, double* uv, double* dist, uint8_t* status,
                           void* ws, size_t ws_bytes, cudaStream_t s);
size_t query_ws_bytes(int64_t n_splines, int64_t n_q);
bspl_status query_curves_learned(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                 const double* q_xyz, const bspl_options* o, int invert, double* t, double* dist,
                                 uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t s);
size_t learned_ws_bytes(int64_t n_splines, int64_t n_q);

// learned seed (mlp.cu)
size_t train_ws_bytes(int64_t batch);

// evaluation (eval.cu)
bspl_status eval_curves(const bspl_curves* c, int64_t n_q, const int32_t* qc, const double* t, double* xyz,
                        cudaStream_t s);
bspl_status eval_surfaces(const bspl_surfaces* c, int64_t n_q, const int32_t* qs, const double* uv, double* xyz,
                          cudaStream_t s);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace bspl
