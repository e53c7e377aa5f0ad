// Batched point projection / inversion on decomposed curves (Sec. 3 Eqs.
// projection, projections, inversion; Sec. 4.2.3 Eqs. Dt, Et, E't; Sec. 4.4.2
// per-query minimum and reparameterisation).
//
// Layout of the work: queries are first grouped by curve (counting sort), then
// one warp takes a batch of 32 consecutive queries.  For each query the warp
// cooperates: lanes stride over the curve's culling groups (32 consecutive
// segments each) for an upper bound of the distance from group reference
// points, then over surviving groups' segments (lower bound = distance to the
// segment's control-point box; upper bound tightened by segment start
// points), then evaluates a grid of S samples on every surviving segment
// (32/S segments per warp step) and detects the sampled basins with
// shuffles.  Every admitted basin goes to a per-warp pool; when the pool
// fills, or the batch ends, each lane runs a safeguarded Newton iteration on
// one pooled basin, so the Newton phase keeps all 32 lanes busy.  The
// per-query minimum is then taken by the lane that owns the query's slot.
//
// Precision: PLAIN runs every stage in FP64 on the FP64 records.  MIXED runs
// culling, grid and the first Newton steps in FP32 on the FP32 records
// (boxes rounded outward, slack on every comparison), then two FP64 Newton
// steps on the FP64 coefficients; a basin whose second FP64 step is not
// below 1e-9 continues with the FP64 safeguarded iteration (FALLBACK).
#include <math.h>

#include "query_common.cuh"

namespace bspl {

namespace {

struct PoolEntry {
    int seg;
    int slot;
    float u0, h;  // h < 0: isolate every minimum of the segment first
};

template <class R>
struct WarpSmem {
    int cand_seg[kCandCap];
    R cand_lb[kCandCap];
    PoolEntry pool[kPoolCap];
    double pool_D[kPoolCap];
    double pool_u[kPoolCap];
    float pool_u32[kPoolCap];  // mixed: FP32 minimiser and its squared distance
    float pool_D32[kPoolCap];
    unsigned char pool_conv32[kPoolCap];  // mixed: the FP32 stage converged
    unsigned char pool_flags[kPoolCap];
    double q64[kQPW][3];
    float q32[kQPW][3];
    float eps32[kQPW];         // mixed: FP32 distance slack of the query
    float best_D32[kQPW];      // mixed: best FP32 squared distance so far
    short fin[kPoolCap];       // mixed: pool entries that get the FP64 finish
    double best_D[kQPW];
    double best_u[kQPW];
    int best_seg[kQPW];
    unsigned char best_flags[kQPW];
};


// Newton phase over the pooled basins, then per-slot merge.
// MIXED: (A) every basin gets FP32 Newton steps; (B) the lane owning each
// query slot takes the best FP32 squared distance; (C) only basins within the
// FP32 error margin of that best (the best one always) get the two FP64
// Newton steps on the FP64 coefficients, with the FP64 safeguarded iteration
// as the fallback when the second step is not below 1e-9.
template <class R, bool MIXED>
__device__ void flush_pool(const CurveQ& P, WarpSmem<R>& W, int npool, int lane, unsigned& it32, unsigned& it64)
{
    if (MIXED) {
        // (A) FP32 refinement in the segment's local frame: the offset
        // a0 - q is formed once in FP64 and rounded, so the FP32 search keeps
        // its relative accuracy on short segments far from the origin
        for (int k = lane; k < npool; k += 32) {
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * e.seg + 6;
            const float* a32 = P.rec32 + (int64_t)BSPL_CREC32 * e.seg + 6;
            float c32[12];
            c32[0] = (float)(a64[0] - q[0]);
            c32[1] = (float)(a64[1] - q[1]);
            c32[2] = (float)(a64[2] - q[2]);
#pragma unroll
            for (int i = 3; i < 12; ++i) c32[i] = a32[i];
            const bool iso = e.h < 0.f;
            float uf = e.u0;
            if (iso) uf = isolate_min<float>(c32, 0.f, 0.f, 0.f, 1e-7f, P.fp32_steps * 4);
            W.pool_conv32[k] =
                newton_min<float>(c32, 0.f, 0.f, 0.f, uf, iso ? 1.f / 64.f : e.h, P.fp32_steps, 1e-7f, it32);
            float E, Ep;
            W.pool_D32[k] = eval_E<float>(c32, 0.f, 0.f, 0.f, uf, E, Ep);
            W.pool_u32[k] = uf;
            W.pool_D[k] = INFINITY;
            W.pool_flags[k] = 0;
        }
        __syncwarp();
        // (B) best FP32 distance per query slot
        if (lane < kQPW) {
            float b = W.best_D32[lane];
            for (int k = 0; k < npool; ++k)
                if (W.pool[k].slot == lane) b = fminf(b, W.pool_D32[k]);
            W.best_D32[lane] = b;
        }
        __syncwarp();
        // (C) compact the entries within the FP32 margin of their query's best
        int nfin = 0;
        for (int base = 0; base < npool; base += 32) {
            const int k = base + lane;
            bool take = false;
            if (k < npool) {
                const int sl = W.pool[k].slot;
                const float sm = sqrtf(W.best_D32[sl]) + 2.f * W.eps32[sl];
                take = !W.pool_conv32[k] || W.pool_D32[k] <= sm * sm;
            }
            const unsigned m = __ballot_sync(kFull, take);
            if (take) W.fin[nfin + __popc(m & ((1u << lane) - 1))] = (short)k;
            nfin += __popc(m);
        }
        __syncwarp();
        // (D) two FP64 Newton steps on the FP64 coefficients, packed over lanes
        for (int f = lane; f < nfin; f += 32) {
            const int k = W.fin[f];
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * e.seg + 6;
            double c64[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) c64[i] = a64[i];
            double u = (double)W.pool_u32[k], last;
            double D = finish64(c64, P.rec32 + (int64_t)BSPL_CREC32 * e.seg + 9, q, u, last, it64);
            unsigned char fl = 0;
            bool ok = last <= 1e-9;
            if (!ok) {
                fl |= BSPL_Q_FALLBACK;
                ok = newton_min<double>(c64, q[0], q[1], q[2], u, e.h < 0.f ? 1.0 / 64 : (double)e.h, P.newton_max,
                                        1e-15, it64);
                double E, Ep;
                D = eval_E(c64, q[0], q[1], q[2], u, E, Ep);
            }
            fl |= ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
            W.pool_D[k] = D;
            W.pool_u[k] = u;
            W.pool_flags[k] = fl;
        }
    } else {
        for (int k = lane; k < npool; k += 32) {
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * e.seg + 6;
            double c64[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) c64[i] = a64[i];
            const bool iso = e.h < 0.f;
            double u = (double)e.u0;
            if (iso) u = isolate_min<double>(c64, q[0], q[1], q[2], 1e-15, P.newton_max);
            bool ok = newton_min<double>(c64, q[0], q[1], q[2], u, iso ? 1.0 / 64 : (double)e.h, P.newton_max,
                                         1e-15, it64);
            double E, Ep;
            W.pool_D[k] = eval_E(c64, q[0], q[1], q[2], u, E, Ep);
            W.pool_u[k] = u;
            W.pool_flags[k] = ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
        }
    }
    __syncwarp();
    if (lane < kQPW) {
        double bD = W.best_D[lane], bu = W.best_u[lane];
        int bs = W.best_seg[lane];
        unsigned char bf = W.best_flags[lane];
        for (int k = 0; k < npool; ++k) {
            if (W.pool[k].slot != lane) continue;
            const double D = W.pool_D[k], u = W.pool_u[k];
            const int sg = W.pool[k].seg;
            if (better(D, sg, u, bD, bs, bu)) {
                bD = D;
                bu = u;
                bs = sg;
                bf = W.pool_flags[k];
            }
        }
        W.best_D[lane] = bD;
        W.best_u[lane] = bu;
        W.best_seg[lane] = bs;
        W.best_flags[lane] = bf;
    }
    __syncwarp();
}

template <class R, int S, bool MIXED, int MINB>
__global__ void __launch_bounds__(kWarps * 32, MINB) k_query_curves(CurveQ P)
{
    __shared__ WarpSmem<R> smem[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<R>& W = smem[wid];
    const int64_t nq = P.n_q_dev ? min(P.n_q, *P.n_q_dev) : P.n_q;
    // persistent: each warp takes batches of 32 sorted queries until none is left
    const int64_t nbatch = (nq + kQPW - 1) / kQPW;
    int round = 0;
    for (int64_t batch = next_batch(P.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round); batch < nbatch;
         batch = next_batch(P.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round)) {
    const int64_t qbase = batch * kQPW;
    const int nslots = (int)min((int64_t)kQPW, nq - qbase);
    const R* rec = Tab<R>::rec(P);
    const R* grp = Tab<R>::grp(P);
    constexpr int RW = Tab<R>::RW, GW = Tab<R>::GW;
    constexpr int SPW = 32 / S;  // segments per grid step
    const R h = R(1) / R(S - 1);
    unsigned long long n_grp_tested = 0, n_seg_tested = 0, n_cand = 0, n_newton = 0;
    unsigned it32 = 0, it64 = 0;  // Newton iterations run by this lane

    if (lane < kQPW) {
        W.best_D[lane] = INFINITY;
        W.best_u[lane] = 0.0;
        W.best_seg[lane] = 0x7fffffff;
        W.best_flags[lane] = 0;
        W.best_D32[lane] = INFINITY;
    }
    int npool = 0;
    __syncwarp();

    for (int sl = 0; sl < nslots; ++sl) {
        const int64_t qi = P.order ? (int64_t)P.order[qbase + sl] : qbase + sl;
        const int c = P.q_curve[qi];
        const double qx64 = P.q_xyz[3 * qi], qy64 = P.q_xyz[3 * qi + 1], qz64 = P.q_xyz[3 * qi + 2];
        const bool bad = c < 0 || c >= P.n || !isfinite(qx64) || !isfinite(qy64) || !isfinite(qz64);
        const R qx = (R)qx64, qy = (R)qy64, qz = (R)qz64;
        const R eps = MIXED ? R(4e-6) * (fabs(qx) + fabs(qy) + fabs(qz) + (R)P.diag[c < 0 || c >= P.n ? 0 : c])
                            : R(1e-13) * (fabs(qx) + fabs(qy) + fabs(qz) + (R)P.diag[c < 0 || c >= P.n ? 0 : c]);
        if (lane == 0) {
            W.q64[sl][0] = qx64;
            W.q64[sl][1] = qy64;
            W.q64[sl][2] = qz64;
            W.q32[sl][0] = (float)qx;
            W.q32[sl][1] = (float)qy;
            W.q32[sl][2] = (float)qz;
            W.eps32[sl] = (float)eps;
            if (bad) W.best_flags[sl] = BSPL_Q_INVALID;
        }
        if (bad) continue;
        const int64_t s0 = P.seg_off[c], s1 = P.seg_off[c + 1];
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];

        // level 1: upper bound from the group reference points
        R ub = INFINITY;
        for (int64_t g = g0 + lane; g < g1; g += 32) ub = fmin(ub, pt_d2(grp + (int64_t)GW * g + 6, qx, qy, qz));
        ub = warp_min(ub);
        R ubs = slacked(ub, eps);
        n_grp_tested += (unsigned long long)(g1 - g0);

        int ncand = 0;
        // grid stage over the buffered candidates
        auto grid_stage = [&]() {
            __syncwarp();
            const int sub = lane / S, j = lane % S;
            for (int base = 0; base < ncand; base += SPW) {
                const int k = base + sub;
                const bool act = k < ncand && W.cand_lb[k] <= ubs;
                const int seg = act ? W.cand_seg[k] : 0;
                R D = INFINITY, spd = 0;
                int nsc = 0;
                const R u = R(j) * h;
                if (act) {
                    R bb[6];
                    nsc = bernstein_E(rec + (int64_t)RW * seg + 6, qx, qy, qz, bb);
                    const R* a = rec + (int64_t)RW * seg + 6;
                    R Dq = 0;
                    const R q3[3] = { qx, qy, qz };
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        R a0 = a[cc], a1 = a[3 + cc], a2 = a[6 + cc], a3 = a[9 + cc];
                        R x = a0 + u * (a1 + u * (a2 + u * a3)) - q3[cc];
                        Dq += x * x;
                        spd += fabs(a1) + R(2) * fabs(a2) + R(3) * fabs(a3);
                    }
                    D = Dq;
                }
                const R Dl = __shfl_up_sync(kFull, D, 1, S);
                const R Dr = __shfl_down_sync(kFull, D, 1, S);
                const bool ismin = act && (j == 0 || D <= Dl) && (j == S - 1 || D < Dr);
                ub = fmin(ub, warp_min(D));
                ubs = slacked(ub, eps);
                // a basin can hold a point within spd*h of its sample; a
                // segment whose E changes sign more than once is handed to
                // the certified isolation instead (one entry, lane j = 0)
                const R adm = slacked(ub, eps + spd * h);
                const bool iso = act && nsc >= 2;
                const bool push = iso ? (j == 0) : (ismin && D <= adm);
                const unsigned m = __ballot_sync(kFull, push);
                const int cnt = __popc(m);
                if (cnt > 0 && npool + cnt > kPoolCap) {
                    flush_pool<R, MIXED>(P, W, npool, lane, it32, it64);
                    n_newton += npool;
                    npool = 0;
                }
                if (push) {
                    const int pos = npool + __popc(m & ((1u << lane) - 1));
                    PoolEntry e;
                    e.seg = seg;
                    e.slot = sl;
                    e.u0 = (float)u;
                    e.h = iso ? -1.f : (float)h;
                    if (j == 0) e.u0 = 0.f;
                    if (j == S - 1) e.u0 = 1.f;
                    W.pool[pos] = e;
                }
                npool += cnt;
                __syncwarp();
            }
            n_cand += (unsigned long long)ncand;
            ncand = 0;
        };

        // level 2: groups that may hold a closer point, then their segments
        for (int64_t gb = g0; gb < g1; gb += 32) {
            const int64_t g = gb + lane;
            const R lbg = g < g1 ? box_d2(grp + (int64_t)GW * g, qx, qy, qz) : R(INFINITY);
            unsigned m = __ballot_sync(kFull, lbg <= ubs);
            while (m) {
                const int jg = __ffs(m) - 1;
                m &= m - 1;
                const R lbj = __shfl_sync(kFull, lbg, jg);
                if (!(lbj <= ubs)) continue;
                const int64_t ss = s0 + (gb + jg - g0) * BSPL_GROUP;
                const int64_t se = min(ss + BSPL_GROUP, s1);
                const int64_t s = ss + lane;
                const bool valid = s < se;
                R lbs = INFINITY, ups = INFINITY;
                if (valid) {
                    const R* r = rec + (int64_t)RW * s;
                    lbs = box_d2(r, qx, qy, qz);
                    ups = pt_d2(r + 6, qx, qy, qz);
                }
                n_seg_tested += (unsigned long long)(se - ss);
                ub = fmin(ub, warp_min(ups));
                ubs = slacked(ub, eps);
                const bool keep = valid && lbs <= ubs;
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) {
                    const int pos = ncand + __popc(km & ((1u << lane) - 1));
                    W.cand_seg[pos] = (int)s;
                    W.cand_lb[pos] = lbs;
                }
                ncand += __popc(km);
                if (ncand > kCandCap - 32) grid_stage();
            }
        }
        grid_stage();
        // the curve's last point (u = 1 of its last segment) is sampled by the
        // grid only when that segment survives; it always survives culling
        // because its start point bounds ub from above only when it is close
        (void)s1;
    }
    if (npool > 0) {
        flush_pool<R, MIXED>(P, W, npool, lane, it32, it64);
        n_newton += npool;
    }
    __syncwarp();

    // write results: lane = slot
    if (lane < nslots) {
        const int64_t qi = P.order ? (int64_t)P.order[qbase + lane] : qbase + lane;
        unsigned char fl = W.best_flags[lane];
        const int seg = W.best_seg[lane];
        if ((fl & BSPL_Q_INVALID) || seg == 0x7fffffff) {
            P.t[qi] = __longlong_as_double(0x7ff8000000000000LL);
            P.dist[qi] = __longlong_as_double(0x7ff8000000000000LL);
            P.status[qi] = BSPL_Q_INVALID;
        } else {
            const double u = W.best_u[lane];
            const double t0 = P.prange[2 * seg], t1 = P.prange[2 * seg + 1];
            const double t = u <= 0.0 ? t0 : (u >= 1.0 ? t1 : t0 + u * (t1 - t0));
            const double d = sqrt(W.best_D[lane]);
            const int c = P.q_curve[qi];
            if ((seg == P.seg_off[c] && u <= 0.0) || (seg == P.seg_off[c + 1] - 1 && u >= 1.0)) fl |= BSPL_Q_AT_END;
            if (P.invert && d > 1e-9 * P.diag[c]) fl |= BSPL_Q_OFF_CURVE;
            P.t[qi] = t;
            P.dist[qi] = d;
            P.status[qi] = fl;
        }
    }
    if (P.counters) {
        unsigned long long fb = 0, nc = 0, i32 = it32, i64 = it64;
        if (lane < nslots) {
            fb = (W.best_flags[lane] & BSPL_Q_FALLBACK) ? 1 : 0;
            nc = (W.best_flags[lane] & BSPL_Q_NONCONV) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fb += __shfl_xor_sync(kFull, fb, o);
            nc += __shfl_xor_sync(kFull, nc, o);
            i32 += __shfl_xor_sync(kFull, i32, o);
            i64 += __shfl_xor_sync(kFull, i64, o);
        }
        if (lane == 0) {
            atomicAdd(P.counters + BSPL_CNT_QUERIES, (unsigned long long)nslots);
            atomicAdd(P.counters + BSPL_CNT_GRP_TESTED, n_grp_tested);
            atomicAdd(P.counters + BSPL_CNT_SEG_TESTED, n_seg_tested);
            atomicAdd(P.counters + BSPL_CNT_CANDIDATES, n_cand);
            atomicAdd(P.counters + BSPL_CNT_NEWTON, n_newton);
            atomicAdd(P.counters + BSPL_CNT_FALLBACK, fb);
            atomicAdd(P.counters + BSPL_CNT_NONCONV, nc);
            atomicAdd(P.counters + BSPL_CNT_NEWTON32_ITERS, i32);
            atomicAdd(P.counters + BSPL_CNT_NEWTON64_ITERS, i64);
        }
    }
    __syncwarp();
    }  // batches
}

// ------------------------------------------------------------ query sorting

// bucket of a query: its spline's rank (heaviest first) or, without ranks,
// its spline index; invalid queries go to the last bucket
__device__ __forceinline__ int64_t sort_bucket(int c, int64_t n, const int32_t* __restrict__ rank)
{
    if (c < 0 || c >= n) return n;
    return rank ? (int64_t)rank[c] : (int64_t)c;
}

__global__ void k_hist(const int32_t* __restrict__ qc, int64_t n_q, int64_t n, const int32_t* __restrict__ rank,
                       int64_t* __restrict__ hist)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q) return;
    atomicAdd((unsigned long long*)(hist + sort_bucket(qc[i], n, rank)), 1ull);
}

__global__ void k_scatter(const int32_t* __restrict__ qc, int64_t n_q, int64_t n, const int32_t* __restrict__ rank,
                          int64_t* __restrict__ cursor, int32_t* __restrict__ order)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q) return;
    unsigned long long pos = atomicAdd((unsigned long long*)(cursor + sort_bucket(qc[i], n, rank)), 1ull);
    order[pos] = (int32_t)i;
}

template <class R, int S, bool MIXED, int MINB>
void launch_query(const CurveQ& P, cudaStream_t s)
{
    int64_t batches = (P.n_q + kQPW - 1) / kQPW;
    int64_t blocks = (batches + kWarps - 1) / kWarps;
    if (P.work) blocks = persistent_blocks(k_query_curves<R, S, MIXED, MINB>, kWarps * 32, 0, blocks);
    k_query_curves<R, S, MIXED, MINB><<<(unsigned)blocks, kWarps * 32, 0, s>>>(P);
}

// occupancy: 0 -> compiler's register choice, 1 -> at least 4 blocks of 4
// warps per SM, 2 -> at least 6 (fewer registers, some spills)
template <class R, int S, bool MIXED>
void launch_occ(const CurveQ& P, int occ, cudaStream_t s)
{
    if (occ == 1) launch_query<R, S, MIXED, 4>(P, s);
    else if (occ == 2) launch_query<R, S, MIXED, 6>(P, s);
    else launch_query<R, S, MIXED, 1>(P, s);
}

}  // namespace

// the mixed-precision grid kernel on the queries listed in P.order (used by
// the learned path for queries whose candidate pairs did not fit)
void launch_mixed_curves(const CurveQ& P, int occ, cudaStream_t s)
{
    launch_occ<float, 16, true>(P, occ, s);
}

size_t query_ws_bytes(int64_t n_splines, int64_t n_q)
{
    Carver cv(nullptr, 0);
    cv.take<int64_t>((size_t)n_splines + 2);
    cv.take<int64_t>(scan_tmp_elems(n_splines + 2));
    cv.take<int32_t>((size_t)n_q);
    cv.take<unsigned long long>(2);
    return cv.used + 256;
}

// groups query indices by spline (heaviest spline first when ranks are
// given): order[] lists queries bucket by bucket; *work receives a zeroed
// counter for the work-stealing launch that follows
cudaError_t sort_by_spline(const int32_t* qc, int64_t n_q, int64_t n, const int32_t* rank, void* ws,
                           size_t ws_bytes, int32_t** order, unsigned long long** work, cudaStream_t s)
{
    Carver cv(ws, ws_bytes);
    int64_t* hist = cv.take<int64_t>((size_t)n + 2);
    int64_t* tmp = cv.take<int64_t>(scan_tmp_elems(n + 2));
    int32_t* ord = cv.take<int32_t>((size_t)n_q);
    unsigned long long* wk = cv.take<unsigned long long>(2);
    if (!hist || !tmp || !ord || !wk) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int64_t) * (size_t)(n + 2), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(wk, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int th = 256;
    k_hist<<<ceil_div(n_q, th), th, 0, s>>>(qc, n_q, n, rank, hist);
    e = exclusive_scan_i64(hist, hist, n + 2, tmp, s);
    if (e != cudaSuccess) return e;
    k_scatter<<<ceil_div(n_q, th), th, 0, s>>>(qc, n_q, n, rank, hist, ord);
    *order = ord;
    if (work) *work = wk;
    return cudaGetLastError();
}

bspl_status query_curves(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve, const double* q_xyz,
                         const bspl_options* opt, int invert, double* t, double* dist, uint8_t* status, void* ws,
                         size_t ws_bytes, cudaStream_t s)
{
    if (!segs || segs->is_surface || n_q < 0) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    if (!q_curve || !q_xyz || !t || !dist || !status || !segs->seg_off || !segs->grp_off || !segs->rec64 ||
        !segs->rec32 || !segs->grp64 || !segs->grp32 || !segs->prange || !segs->diag)
        return BSPL_EINVAL;
    if (n_q > 0x7fffffffLL || segs->capacity > 0x7fffffffLL) return BSPL_EINVAL;
    bspl_options o{};
    if (opt) o = *opt;
    int samples = o.samples ? o.samples : 16;
    if (samples != 8 && samples != 16 && samples != 32) return BSPL_EINVAL;
    if (o.prec == BSPL_LEARNED_MIXED || o.prec == BSPL_CLIP_MIXED)
        return query_curves_learned(segs, n_q, q_curve, q_xyz, &o, invert, t, dist, status, ws, ws_bytes, s);
    if (o.prec != BSPL_FP64 && o.prec != BSPL_MIXED) return BSPL_EINVAL;
    int sort = opt ? o.sort_queries : 1;
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
    P.order = nullptr;
    if (sort) {
        if (!ws || ws_bytes < query_ws_bytes(segs->n, n_q)) return BSPL_EINVAL;
        int32_t* ord = nullptr;
        if (sort_by_spline(q_curve, n_q, segs->n, segs->spline_rank, ws, ws_bytes, &ord, &P.work, s) !=
            cudaSuccess)
            return BSPL_ECUDA;
        P.order = ord;
    }
    const bool mixed = o.prec == BSPL_MIXED;
    const int occ = o.occupancy;
    if (occ < 0 || occ > 2) return BSPL_EINVAL;
    if (mixed) {
        if (samples == 8) launch_query<float, 8, true, 1>(P, s);
        else if (samples == 16) launch_occ<float, 16, true>(P, occ, s);
        else launch_occ<float, 32, true>(P, occ, s);
    } else {
        if (samples == 8) launch_query<double, 8, false, 1>(P, s);
        else if (samples == 16) launch_occ<double, 16, false>(P, occ, s);
        else launch_occ<double, 32, false>(P, occ, s);
    }
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl
