// Scratch-free variant of the curve projection entry point: the workspace
// is a fixed array in device memory owned by the library instead of a
// caller allocation.  See bspl_project_curves_noalloc in include/bspl.h.
#include <mutex>

#include "bspl_internal.cuh"

namespace {

constexpr size_t kScratchBytes = BSPL_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Device-side scratch; in host code this name only stands for the array,
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_addr[kMaxDevices];

// device address of g_scratch on the current device (looked up once per device)
bspl_status scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSPL_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return BSPL_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return BSPL_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return BSPL_OK;
}

}  // namespace

extern "C" bspl_status bspl_project_curves_noalloc(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                                   const double* q_xyz, const bspl_options* opt, double* t,
                                                   double* dist, uint8_t* status, cudaStream_t stream)
{
    if (!segs || n_q < 0) return BSPL_EINVAL;
    if (n_q > BSPL_NOALLOC_MAX_QUERIES || segs->n > BSPL_NOALLOC_MAX_SPLINES) return BSPL_ENOSPACE;
    if (bspl::query_ws_bytes(segs->n, n_q) > kScratchBytes) return BSPL_ENOSPACE;
    // the learned precision adds its culling-candidate and pair buffers
    // (about 1.4 KB per query), so it fits far fewer queries into the array
    if (opt && (opt->prec == BSPL_LEARNED_MIXED || opt->prec == BSPL_CLIP_MIXED) &&
        bspl::learned_ws_bytes(segs->n, n_q) > kScratchBytes)
        return BSPL_ENOSPACE;
    void* ws = nullptr;
    bspl_status st = scratch_address(&ws);
    if (st != BSPL_OK) return st;
    return bspl::query_curves(segs, n_q, q_curve, q_xyz, opt, 0, t, dist, status, ws, kScratchBytes, stream);
}
