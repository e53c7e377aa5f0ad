// Curve projection / inversion with the learned Newton seed (bspl_mlp.h).
//
// Pipeline (one stream, no host synchronisation):
//   1. k_cull_pairs: queries grouped by curve, one warp per 32 queries, the
//      same two-level box culling as the grid kernel.  Every surviving
//      (query, segment) pair is classified by the signs of the Bernstein
//      coefficients of E = (C - q).C' (degree 5, the T matrix of Sec. 4.3),
//      each coefficient compared with a bound on its FP32 rounding error:
//        one sign change, E(0) < 0 < E(1)  -> exactly one minimum inside:
//                                             SEED (the network's job);
//        no sign change                     -> minimum at u = 0 or u = 1;
//        one change, E(0) > 0 > E(1)        -> a maximum inside: the smaller
//                                             end;
//        more changes, or a coefficient within its rounding bound of 0
//                                           -> certified isolation (ISO).
//      Pairs go to one buffer: seeds from the front, the others from the
//      back, so the network reads a dense range.
//   2. the fused MLP (mlp.cu) writes the seed u0 of every SEED pair (without
//      a network: u0 = 1/2).
//   3. one thread per pair: FP32 Newton in the segment's local frame
//      (bracketed by the known sign change for SEED pairs), per-query
//      minimum of the FP32 distances by an integer atomicMin on the float
//      bits; then the two FP64 Newton steps (and the FP64 safeguarded
//      iteration when the second step is not below 1e-9) for the pairs within
//      the FP32 error margin of their query's best; then the per-query
//      lexicographic minimum over (D, segment) by two more atomicMin passes,
//      and the unique winning pair writes the result (Sec. 4.4.2).
//   4. queries whose pairs did not fit the buffer run through the grid
//      kernel (mixed precision) over a device-side list.
#include "../../include/bspl_mlp.h"
#include "query_common.cuh"

namespace bspl {

cudaError_t mlp_seed_pairs(const bspl_mlp* m, const int32_t* pq, const int32_t* ps, const double* q_xyz,
                           const bspl_segments* segs, int64_t cap, const unsigned long long* n_dev, float* u0,
                           cudaStream_t s);

namespace {

enum : uint8_t { kSeed = 0, kEnd0 = 1, kEnd1 = 2, kEnds = 3, kIso = 4 };
constexpr int kPairsPerQuery = 24;  // buffer capacity per query

struct PairBuf {
    int32_t* pq;
    int32_t* ps;
    uint8_t* kind;
    float* u;
    float* D32;
    uint8_t* conv;
    double* D64;
    double* u64;
    uint8_t* fl;
    int64_t cap;
    unsigned long long* cnt;  // [0] reserved, [1] seeds, [2] others, [3] overflowed queries
    int32_t* over;            // overflowed query indices
    unsigned* best32;         // per query: FP32 distance bits
    unsigned long long* best64;
    int* bestseg;
};

// classification of a pair from its FP32 local-frame cubic c (C - q)
__device__ __forceinline__ uint8_t classify(const float* c)
{
    float e[6] = { 0, 0, 0, 0, 0, 0 }, ea[6] = { 0, 0, 0, 0, 0, 0 };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float c0 = c[k], c1 = c[3 + k], c2 = c[6 + k], c3 = c[9 + k];
        const float d1 = c1, d2 = 2.f * c2, d3 = 3.f * c3;
        e[0] += c0 * d1;
        e[1] += c0 * d2 + c1 * d1;
        e[2] += c0 * d3 + c1 * d2 + c2 * d1;
        e[3] += c1 * d3 + c2 * d2 + c3 * d1;
        e[4] += c2 * d3 + c3 * d2;
        e[5] += c3 * d3;
        const float a0 = fabsf(c0), a1 = fabsf(c1), a2 = fabsf(c2), a3 = fabsf(c3);
        ea[0] += a0 * a1;
        ea[1] += 2.f * a0 * a2 + a1 * a1;
        ea[2] += 3.f * a0 * a3 + 3.f * a1 * a2;
        ea[3] += 4.f * a1 * a3 + 2.f * a2 * a2;
        ea[4] += 5.f * a2 * a3;
        ea[5] += 3.f * a3 * a3;
    }
    float b[6], ba[6];
    b[0] = e[0];
    b[1] = e[0] + 0.2f * e[1];
    b[2] = e[0] + 0.4f * e[1] + 0.1f * e[2];
    b[3] = e[0] + 0.6f * e[1] + 0.3f * e[2] + 0.1f * e[3];
    b[4] = e[0] + 0.8f * e[1] + 0.6f * e[2] + 0.4f * e[3] + 0.2f * e[4];
    b[5] = e[0] + e[1] + e[2] + e[3] + e[4] + e[5];
    ba[0] = ea[0];
    ba[1] = ea[0] + 0.2f * ea[1];
    ba[2] = ea[0] + 0.4f * ea[1] + 0.1f * ea[2];
    ba[3] = ea[0] + 0.6f * ea[1] + 0.3f * ea[2] + 0.1f * ea[3];
    ba[4] = ea[0] + 0.8f * ea[1] + 0.6f * ea[2] + 0.4f * ea[3] + 0.2f * ea[4];
    ba[5] = ea[0] + ea[1] + ea[2] + ea[3] + ea[4] + ea[5];
    int v = 0, last = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float tol = 1e-5f * ba[i];
        const int s = b[i] > tol ? 1 : (b[i] < -tol ? -1 : 0);
        if (s == 0) return kIso;
        if (last != 0 && s != last) ++v;
        last = s;
    }
    const bool neg0 = b[0] < 0.f;
    if (v == 0) return neg0 ? kEnd1 : kEnd0;
    if (v == 1) return neg0 ? kSeed : kEnds;
    return kIso;
}

__device__ __forceinline__ void local32(const CurveQ& P, int64_t seg, const double* q, float* c)
{
    const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * seg + 6;
    const float* a32 = P.rec32 + (int64_t)BSPL_CREC32 * seg + 6;
    c[0] = (float)(a64[0] - q[0]);
    c[1] = (float)(a64[1] - q[1]);
    c[2] = (float)(a64[2] - q[2]);
#pragma unroll
    for (int i = 3; i < 12; ++i) c[i] = a32[i];
}

template <bool SEEDS_ONLY>
__global__ void __launch_bounds__(kWarps * 32) k_cull_pairs(CurveQ P, PairBuf B)
{
    __shared__ int s_seg[kWarps][kCandCap];
    __shared__ float s_lb[kWarps][kCandCap];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* cseg = s_seg[wid];
    float* clb = s_lb[wid];
    const int64_t qbase = ((int64_t)blockIdx.x * kWarps + wid) * kQPW;
    if (qbase >= P.n_q) return;
    const int nslots = (int)min((int64_t)kQPW, P.n_q - qbase);
    const float* rec = P.rec32;
    const float* grp = P.grp32;
    constexpr int RW = BSPL_CREC32, GW = BSPL_GREC32;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long n_grp = 0, n_seg = 0, n_pairs = 0;

    for (int sl = 0; sl < nslots; ++sl) {
        const int64_t qi = P.order ? (int64_t)P.order[qbase + sl] : qbase + sl;
        const int c = P.q_curve[qi];
        const double q64[3] = { P.q_xyz[3 * qi], P.q_xyz[3 * qi + 1], P.q_xyz[3 * qi + 2] };
        const bool bad = c < 0 || c >= P.n || !isfinite(q64[0]) || !isfinite(q64[1]) || !isfinite(q64[2]);
        if (bad) {
            if (!SEEDS_ONLY && lane == 0) {
                P.t[qi] = __longlong_as_double(0x7ff8000000000000LL);
                P.dist[qi] = __longlong_as_double(0x7ff8000000000000LL);
                P.status[qi] = BSPL_Q_INVALID;
            }
            continue;
        }
        if (!SEEDS_ONLY && lane == 0) {
            B.best32[qi] = 0x7f800000u;
            B.best64[qi] = 0x7ff0000000000000ull;
            B.bestseg[qi] = 0x7fffffff;
            P.t[qi] = __longlong_as_double(0x7ff8000000000000LL);
            P.dist[qi] = __longlong_as_double(0x7ff8000000000000LL);
            P.status[qi] = BSPL_Q_NONCONV;
        }
        const float qx = (float)q64[0], qy = (float)q64[1], qz = (float)q64[2];
        const float eps = 4e-6f * (fabsf(qx) + fabsf(qy) + fabsf(qz) + (float)P.diag[c]);
        const int64_t s0 = P.seg_off[c], s1 = P.seg_off[c + 1];
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];
        float ub = INFINITY;
        for (int64_t g = g0 + lane; g < g1; g += 32) ub = fminf(ub, pt_d2(grp + (int64_t)GW * g + 6, qx, qy, qz));
        ub = warp_min(ub);
        float ubs = slacked(ub, eps);
        n_grp += (unsigned long long)(g1 - g0);
        int ncand = 0;
        bool overflow = false;
        auto emit = [&]() {
            __syncwarp();
            for (int base = 0; base < ncand; base += 32) {
                const int k = base + lane;
                const bool act = k < ncand && clb[k] <= ubs;
                const int seg = act ? cseg[k] : 0;
                uint8_t kind = kIso;
                if (act) {
                    float cl[12];
                    local32(P, seg, q64, cl);
                    kind = classify(cl);
                }
                const bool is_seed = act && kind == kSeed;
                const bool is_oth = !SEEDS_ONLY && act && kind != kSeed;
                const unsigned ms = __ballot_sync(kFull, is_seed), mo = __ballot_sync(kFull, is_oth);
                const int cs = __popc(ms), co = __popc(mo);
                if (cs + co == 0) continue;
                unsigned long long bs = 0, bo = 0;
                int ok = 0;
                if (lane == 0) {
                    const unsigned long long tot = atomicAdd(B.cnt, (unsigned long long)(cs + co));
                    ok = tot + cs + co <= (unsigned long long)B.cap;
                    if (ok) {
                        bs = cs ? atomicAdd(B.cnt + 1, (unsigned long long)cs) : 0;
                        bo = co ? atomicAdd(B.cnt + 2, (unsigned long long)co) : 0;
                    }
                }
                ok = __shfl_sync(kFull, ok, 0);
                bs = __shfl_sync(kFull, bs, 0);
                bo = __shfl_sync(kFull, bo, 0);
                if (!ok) {
                    overflow = true;
                    continue;
                }
                if (lane == 0) n_pairs += (unsigned long long)(cs + co);
                if (is_seed) {
                    const int64_t idx = (int64_t)bs + __popc(ms & lt);
                    B.pq[idx] = (int32_t)qi;
                    B.ps[idx] = seg;
                    if (B.kind) B.kind[idx] = kSeed;
                }
                if (is_oth) {
                    const int64_t idx = B.cap - 1 - ((int64_t)bo + __popc(mo & lt));
                    B.pq[idx] = (int32_t)qi;
                    B.ps[idx] = seg;
                    B.kind[idx] = kind;
                }
            }
            ncand = 0;
            __syncwarp();
        };
        for (int64_t gb = g0; gb < g1; gb += 32) {
            const int64_t g = gb + lane;
            const float lbg = g < g1 ? box_d2(grp + (int64_t)GW * g, qx, qy, qz) : INFINITY;
            unsigned m = __ballot_sync(kFull, lbg <= ubs);
            while (m) {
                const int jg = __ffs(m) - 1;
                m &= m - 1;
                const float lbj = __shfl_sync(kFull, lbg, jg);
                if (!(lbj <= ubs)) continue;
                const int64_t ss = s0 + (gb + jg - g0) * BSPL_GROUP;
                const int64_t se = min(ss + BSPL_GROUP, s1);
                const int64_t s = ss + lane;
                const bool valid = s < se;
                float lbs = INFINITY, ups = INFINITY;
                if (valid) {
                    const float* r = rec + (int64_t)RW * s;
                    lbs = box_d2(r, qx, qy, qz);
                    ups = pt_d2(r + 6, qx, qy, qz);
                }
                n_seg += (unsigned long long)(se - ss);
                ub = fminf(ub, warp_min(ups));
                ubs = slacked(ub, eps);
                const bool keep = valid && lbs <= ubs;
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) {
                    const int pos = ncand + __popc(km & lt);
                    cseg[pos] = (int)s;
                    clb[pos] = lbs;
                }
                ncand += __popc(km);
                if (ncand > kCandCap - 32) emit();
            }
        }
        emit();
        if (!SEEDS_ONLY && overflow && lane == 0) {
            const unsigned long long pos = atomicAdd(B.cnt + 3, 1ull);
            B.over[pos] = (int32_t)qi;
        }
    }
    if (!SEEDS_ONLY && P.counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n_pairs += __shfl_xor_sync(kFull, n_pairs, o);
        if (lane == 0) {
            atomicAdd(P.counters + BSPL_CNT_QUERIES, (unsigned long long)nslots);
            atomicAdd(P.counters + BSPL_CNT_GRP_TESTED, n_grp);
            atomicAdd(P.counters + BSPL_CNT_SEG_TESTED, n_seg);
            atomicAdd(P.counters + BSPL_CNT_CANDIDATES, n_pairs);
        }
    }
}

// pair index j in [0, seeds + others) -> buffer slot
__device__ __forceinline__ int64_t pair_slot(const PairBuf& B, int64_t j, int64_t ns)
{
    return j < ns ? j : B.cap - 1 - (j - ns);
}

__device__ __forceinline__ void add_counter(unsigned long long* ctr, int which, unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr + which, v);
}

// (3a) FP32 solve of every pair, per-query FP32 minimum
__global__ void k_pairs_fp32(CurveQ P, PairBuf B, int have_seed)
{
    const int64_t ns = (int64_t)B.cnt[1], no = (int64_t)B.cnt[2], np = ns + no;
    unsigned it32 = 0;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < np; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        if (j < np) {
            const int64_t i = pair_slot(B, j, ns);
            const int64_t qi = B.pq[i], seg = B.ps[i];
            const uint8_t kind = j < ns ? kSeed : B.kind[i];
            const double* q = P.q_xyz + 3 * qi;
            float c[12];
            local32(P, seg, q, c);
            float u, E, Ep;
            bool conv = true;
            if (kind == kSeed) {
                float lo = 0.f, hi = 1.f;
                u = have_seed ? fminf(fmaxf(B.u[i], 0.f), 1.f) : 0.5f;
                conv = false;
                for (int it = 0; it < 3 * P.fp32_steps; ++it) {
                    ++it32;
                    eval_E<float>(c, 0.f, 0.f, 0.f, u, E, Ep);
                    if (E > 0.f) hi = u;
                    else if (E < 0.f) lo = u;
                    else {
                        conv = true;
                        break;
                    }
                    float un = Ep > 0.f ? u - E / Ep : 0.5f * (lo + hi);
                    if (Ep > 0.f && fabsf(un - u) <= 1e-7f) {  // converged (the step may round onto lo or hi)
                        u = fminf(fmaxf(un, lo), hi);
                        conv = true;
                        break;
                    }
                    if (!(un > lo && un < hi)) un = 0.5f * (lo + hi);
                    const float mv = fabsf(un - u);
                    u = un;
                    if (mv <= 1e-7f || hi - lo <= 1e-7f) {
                        conv = true;
                        break;
                    }
                }
            } else if (kind == kEnd0) u = 0.f;
            else if (kind == kEnd1) u = 1.f;
            else if (kind == kEnds) {
                const float D0 = eval_E<float>(c, 0.f, 0.f, 0.f, 0.f, E, Ep);
                const float D1 = eval_E<float>(c, 0.f, 0.f, 0.f, 1.f, E, Ep);
                u = D1 < D0 ? 1.f : 0.f;
            } else {
                u = isolate_min<float>(c, 0.f, 0.f, 0.f, 1e-7f, P.fp32_steps * 4);
                conv = newton_min<float>(c, 0.f, 0.f, 0.f, u, 1.f / 64.f, P.fp32_steps, 1e-7f, it32);
            }
            const float D = eval_E<float>(c, 0.f, 0.f, 0.f, u, E, Ep);
            B.u[i] = u;
            B.D32[i] = D;
            B.conv[i] = conv ? 1 : 0;
            atomicMin(B.best32 + qi, __float_as_uint(D));
        }
    }
    if (P.counters) add_counter(P.counters, BSPL_CNT_NEWTON32_ITERS, it32);
}

// (3b) FP64 finish of the pairs within the FP32 margin of their query's best
__global__ void k_pairs_fp64(CurveQ P, PairBuf B)
{
    const int64_t ns = (int64_t)B.cnt[1], no = (int64_t)B.cnt[2], np = ns + no;
    unsigned it64 = 0, nfin = 0;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < np; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        if (j < np) {
            const int64_t i = pair_slot(B, j, ns);
            const int64_t qi = B.pq[i], seg = B.ps[i];
            const double* q = P.q_xyz + 3 * qi;
            const float qx = (float)q[0], qy = (float)q[1], qz = (float)q[2];
            const float eps = 4e-6f * (fabsf(qx) + fabsf(qy) + fabsf(qz) + (float)P.diag[P.q_curve[qi]]);
            const float sm = sqrtf(__uint_as_float(B.best32[qi])) + 2.f * eps;
            if (B.conv[i] && B.D32[i] > sm * sm) {
                B.D64[i] = INFINITY;
                continue;
            }
            ++nfin;
            const uint8_t kind = j < ns ? kSeed : B.kind[i];
            const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * seg + 6;
            double c64[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) c64[k] = a64[k];
            double u = (double)B.u[i], last = 1.0, E, Ep;
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                ++it64;
                eval_E(c64, q[0], q[1], q[2], u, E, Ep);
                double un = Ep > 0.0 ? u - E / Ep : u;
                un = fmin(fmax(un, 0.0), 1.0);
                last = fabs(un - u);
                u = un;
            }
            uint8_t fl = 0;
            bool ok = last <= 1e-9;
            if (!ok) {
                fl |= BSPL_Q_FALLBACK;
                ok = newton_min<double>(c64, q[0], q[1], q[2], u, kind == kIso ? 1.0 / 64 : 0.25, P.newton_max, 1e-15,
                                        it64);
            }
            fl |= ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
            const double D = eval_E(c64, q[0], q[1], q[2], u, E, Ep);
            B.D64[i] = D;
            B.u64[i] = u;
            B.fl[i] = fl;
            atomicMin(B.best64 + qi, (unsigned long long)__double_as_longlong(D));
        }
    }
    if (P.counters) {
        add_counter(P.counters, BSPL_CNT_NEWTON64_ITERS, it64);
        add_counter(P.counters, BSPL_CNT_NEWTON, nfin);
    }
}

// (3c) smallest segment among the pairs at the query's best FP64 distance
__global__ void k_pairs_argseg(CurveQ P, PairBuf B)
{
    const int64_t ns = (int64_t)B.cnt[1], np = ns + (int64_t)B.cnt[2];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = pair_slot(B, j, ns);
        const int64_t qi = B.pq[i];
        if ((unsigned long long)__double_as_longlong(B.D64[i]) == B.best64[qi]) atomicMin(B.bestseg + qi, B.ps[i]);
    }
}

// (3d) the winning pair writes its query's result
__global__ void k_pairs_write(CurveQ P, PairBuf B)
{
    const int64_t ns = (int64_t)B.cnt[1], np = ns + (int64_t)B.cnt[2];
    unsigned fb = 0, nc = 0;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < np; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        if (j < np) {
            const int64_t i = pair_slot(B, j, ns);
            const int64_t qi = B.pq[i];
            const int seg = B.ps[i];
            if ((unsigned long long)__double_as_longlong(B.D64[i]) != B.best64[qi] || seg != B.bestseg[qi]) continue;
            const double u = B.u64[i];
            const double t0 = P.prange[2 * seg], t1 = P.prange[2 * seg + 1];
            const double t = u <= 0.0 ? t0 : (u >= 1.0 ? t1 : t0 + u * (t1 - t0));
            const double d = sqrt(B.D64[i]);
            const int c = P.q_curve[qi];
            unsigned char fl = B.fl[i];
            if ((seg == P.seg_off[c] && u <= 0.0) || (seg == P.seg_off[c + 1] - 1 && u >= 1.0)) fl |= BSPL_Q_AT_END;
            if (P.invert && d > 1e-9 * P.diag[c]) fl |= BSPL_Q_OFF_CURVE;
            P.t[qi] = t;
            P.dist[qi] = d;
            P.status[qi] = fl;
            fb += (fl & BSPL_Q_FALLBACK) ? 1 : 0;
            nc += (fl & BSPL_Q_NONCONV) ? 1 : 0;
        }
    }
    if (P.counters) {
        add_counter(P.counters, BSPL_CNT_FALLBACK, fb);
        add_counter(P.counters, BSPL_CNT_NONCONV, nc);
    }
}

int64_t pair_cap(int64_t n_q) { return kPairsPerQuery * n_q + 4096; }

struct LearnedWs {
    int32_t* order;  // from the sort (inside the sort's own carve)
    PairBuf B;
};

// carve: [sort workspace][pair buffers][per-query arrays][counters]
bool carve_learned(void* ws, size_t bytes, int64_t n_splines, int64_t n_q, PairBuf& B, void** sort_ws,
                   size_t* sort_bytes, size_t* total)
{
    const size_t sb = query_ws_bytes(n_splines, n_q);
    Carver cv(ws, bytes);
    char* sw = cv.take<char>(sb);
    const int64_t cap = pair_cap(n_q);
    B.cap = cap;
    B.pq = cv.take<int32_t>((size_t)cap);
    B.ps = cv.take<int32_t>((size_t)cap);
    B.kind = cv.take<uint8_t>((size_t)cap);
    B.u = cv.take<float>((size_t)cap);
    B.D32 = cv.take<float>((size_t)cap);
    B.conv = cv.take<uint8_t>((size_t)cap);
    B.D64 = cv.take<double>((size_t)cap);
    B.u64 = cv.take<double>((size_t)cap);
    B.fl = cv.take<uint8_t>((size_t)cap);
    B.over = cv.take<int32_t>((size_t)n_q);
    B.best32 = cv.take<unsigned>((size_t)n_q);
    B.best64 = cv.take<unsigned long long>((size_t)n_q);
    B.bestseg = cv.take<int>((size_t)n_q);
    B.cnt = cv.take<unsigned long long>(4);
    if (sort_ws) *sort_ws = sw;
    if (sort_bytes) *sort_bytes = sb;
    if (total) *total = cv.used + 256;
    return ws != nullptr && cv.used <= bytes && B.cnt != nullptr;
}

CurveQ make_params(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                   const bspl_options& o, int invert, double* t, double* dist, uint8_t* status)
{
    CurveQ P{};
    P.seg_off = segs->seg_off;
    P.grp_off = segs->grp_off;
    P.rec64 = segs->rec64;
    P.rec32 = segs->rec32;
    P.grp64 = segs->grp64;
    P.grp32 = segs->grp32;
    P.prange = segs->prange;
    P.diag = segs->diag;
    P.n = segs->n;
    P.n_q = n_q;
    P.q_curve = q_curve;
    P.q_xyz = q_xyz;
    P.t = t;
    P.dist = dist;
    P.status = status;
    P.invert = invert;
    P.newton_max = o.newton_max > 0 ? o.newton_max : 30;
    P.fp32_steps = o.fp32_steps > 0 ? o.fp32_steps : 4;
    P.counters = (unsigned long long*)o.counters;
    return P;
}

bool segs_ok(const bspl_segments* segs)
{
    return segs && !segs->is_surface && segs->seg_off && segs->grp_off && segs->rec64 && segs->rec32 &&
           segs->grp64 && segs->grp32 && segs->prange && segs->diag && segs->capacity <= 0x7fffffffLL;
}

int pair_grid()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (nsm > 0 ? nsm : 1) * 8;
}

}  // namespace

size_t learned_ws_bytes(int64_t n_splines, int64_t n_q)
{
    PairBuf B{};
    size_t total = 0;
    carve_learned(nullptr, 0, n_splines, n_q, B, nullptr, nullptr, &total);
    return total;
}

bspl_status query_curves_learned(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                                 const bspl_options* o, int invert, double* t, double* dist, uint8_t* status,
                                 void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!segs_ok(segs) || n_q < 0 || n_q > 0x7fffffffLL) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    if (!q_curve || !q_xyz || !t || !dist || !status) return BSPL_EINVAL;
    const bspl_mlp* mlp = (const bspl_mlp*)o->mlp;
    if (mlp && (!mlp->params || !mlp->wbf16)) return BSPL_EINVAL;
    if (o->occupancy < 0 || o->occupancy > 2) return BSPL_EINVAL;
    PairBuf B{};
    void* sw = nullptr;
    size_t sb = 0;
    if (!carve_learned(ws, ws_bytes, segs->n, n_q, B, &sw, &sb, nullptr)) return BSPL_EINVAL;
    CurveQ P = make_params(segs, n_q, q_curve, q_xyz, *o, invert, t, dist, status);
    const cudaEvent_t* ev = (const cudaEvent_t*)o->stage_events;
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], s);
    };
    mark(0);
    int32_t* order = nullptr;
    if (sort_by_spline(q_curve, n_q, segs->n, sw, sb, &order, s) != cudaSuccess) return BSPL_ECUDA;
    P.order = order;
    if (cudaMemsetAsync(B.cnt, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) return BSPL_ECUDA;
    mark(1);
    const int64_t blocks = (n_q + kQPW * kWarps - 1) / (kQPW * kWarps);
    k_cull_pairs<false><<<(unsigned)blocks, kWarps * 32, 0, s>>>(P, B);
    mark(2);
    if (mlp && mlp_seed_pairs(mlp, B.pq, B.ps, q_xyz, segs, B.cap, B.cnt + 1, B.u, s) != cudaSuccess)
        return BSPL_ECUDA;
    mark(3);
    const int grid = pair_grid();
    k_pairs_fp32<<<grid, 256, 0, s>>>(P, B, mlp ? 1 : 0);
    mark(4);
    k_pairs_fp64<<<grid, 256, 0, s>>>(P, B);
    mark(5);
    k_pairs_argseg<<<grid, 256, 0, s>>>(P, B);
    k_pairs_write<<<grid, 256, 0, s>>>(P, B);
    mark(6);
    // queries whose pairs did not fit: the grid kernel over the device-side list
    CurveQ F = P;
    F.order = B.over;
    F.n_q_dev = reinterpret_cast<const int64_t*>(B.cnt + 3);
    F.counters = nullptr;
    launch_mixed_curves(F, o->occupancy, s);
    mark(7);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl

using namespace bspl;

extern "C" bspl_status bspl_mlp_collect_pairs(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                              const double* q_xyz, int64_t cap, int32_t* pair_q, int32_t* pair_seg,
                                              int64_t* n_pairs, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!segs_ok(segs) || n_q < 0 || n_q > 0x7fffffffLL || cap < 0 || !n_pairs) return BSPL_EINVAL;
    if (n_q > 0 && (!q_curve || !q_xyz || (cap > 0 && (!pair_q || !pair_seg)))) return BSPL_EINVAL;
    PairBuf B{};
    void* sw = nullptr;
    size_t sb = 0;
    if (!carve_learned(ws, ws_bytes, segs->n, n_q, B, &sw, &sb, nullptr)) return BSPL_EINVAL;
    if (cudaMemsetAsync(B.cnt, 0, 4 * sizeof(unsigned long long), stream) != cudaSuccess) return BSPL_ECUDA;
    if (n_q > 0) {
        bspl_options o{};
        CurveQ P = make_params(segs, n_q, q_curve, q_xyz, o, 0, nullptr, nullptr, nullptr);
        P.counters = nullptr;
        int32_t* order = nullptr;
        if (sort_by_spline(q_curve, n_q, segs->n, sw, sb, &order, stream) != cudaSuccess) return BSPL_ECUDA;
        P.order = order;
        PairBuf C = B;
        C.pq = pair_q;
        C.ps = pair_seg;
        C.kind = nullptr;
        C.cap = cap;
        const int64_t blocks = (n_q + kQPW * kWarps - 1) / (kQPW * kWarps);
        k_cull_pairs<true><<<(unsigned)blocks, kWarps * 32, 0, stream>>>(P, C);
    }
    if (cudaMemcpyAsync(n_pairs, B.cnt, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return BSPL_ECUDA;
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}
