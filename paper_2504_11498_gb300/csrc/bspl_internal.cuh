// Internal declarations shared by the CUDA translation units of libbspl.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bspl.h"

namespace bspl {

constexpr int kMaxCurveDegree = 63;
// highest degree whose spans are extracted by the matrix route (Eq.
// decomfinal): its FP64 error against knot insertion grows about tenfold
// every two degrees (6e-14 of the control points' size at degree 7, 2e-10
// at 15, 1e-2 at 31); above, the blossom
constexpr int kMatrixMaxDeg = 7;
constexpr int kEvalMidDeg = 31;  // the evaluation's and refinement's instances: up to 31, up to 63
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

// workspaces are carved at 256-byte offsets from their start, which must
// itself be 256-byte aligned (as cudaMalloc returns)
inline bool ws_misaligned(const void* ws) { return ws != nullptr && ((uintptr_t)ws & 255u) != 0; }

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
// counting sort of query indices by spline (query_curves.cu): order[] lists
// the queries bucket by bucket (heaviest spline first when ranks are given,
// else by spline index); *work (when asked for) receives a zeroed counter
cudaError_t sort_by_spline(const int32_t* qc, int64_t n_q, int64_t n, const int32_t* rank, void* ws,
                           size_t ws_bytes, int32_t** order, unsigned long long** work, cudaStream_t s);
bspl_status query_curves_learned(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                 const double* q_xyz, const bspl_options* o, int invert, double* t, double* dist,
                                 uint8_t* status, void* ws, size_t ws_bytes, cudaStream_t s);
size_t learned_ws_bytes(int64_t n_splines, int64_t n_q);
size_t learned_surf_ws_bytes(int64_t n_splines, int64_t n_q);

// learned seed (mlp.cu)
size_t train_ws_bytes(int kind, int64_t batch);

// evaluation (eval.cu)
bspl_status eval_curves(const bspl_curves* c, int64_t n_q, const int32_t* qc, const double* t, double* xyz,
                        cudaStream_t s);
bspl_status eval_surfaces(const bspl_surfaces* c, int64_t n_q, const int32_t* qs, const double* uv, double* xyz,
                          cudaStream_t s);
size_t refine_ws_bytes(int64_t n_splines, int64_t n_cp_total, int64_t n_q);
bspl_status refine_curves(const bspl_curves* c, const double* diag, int invert, int64_t n_q, const int32_t* qc,
                          const double* q_xyz, int max_iter, double* t, double* dist, uint8_t* status,
                          uint64_t* evals, void* ws, size_t ws_bytes, cudaStream_t s);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Blocks of a persistent, work-stealing launch: as many as can be resident
// on the GPU at once (SMs x blocks per SM for this kernel, threads and
// dynamic shared memory), but no more than the batches need.
template <class K>
inline int persistent_blocks(K kernel, int threads, size_t smem, int64_t blocks_needed)
{
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    const int64_t g = (int64_t)(nsm > 0 ? nsm : 1) * (occ > 0 ? occ : 1);
    return (int)(blocks_needed < g ? (blocks_needed > 0 ? blocks_needed : 1) : g);
}

// The next batch of a warp in a work-stealing launch: lane 0 takes it from
// the counter (each batch is handed out once; the counter only grows, so the
// loop that calls this ends once it passes the batch count).  Without a
// counter the warp takes its own batch once.
__device__ __forceinline__ int64_t next_batch(unsigned long long* work, int64_t own, int64_t nbatch, int& round)
{
    if (!work) return round++ == 0 ? own : nbatch;
    unsigned long long b = 0;
    if ((threadIdx.x & 31) == 0) b = atomicAdd(work, 1ull);
    return (int64_t)__shfl_sync(0xffffffffu, b, 0);
}

}  // namespace bspl
