// Curve projection / inversion with the learned Newton seed (bspl_mlp.h).
//
// Pipeline (one stream, no host synchronisation):
//   1. k_cull_cands: queries grouped by curve, one warp per 32 queries, the
//      same two-level box culling as the grid kernel; the surviving (query,
//      segment) candidates and each query's final upper bound go to global
//      memory.  k_classify, one thread per candidate: every candidate whose
//      box still passes its query's bound is classified by the signs of the
//      Bernstein coefficients of E = (C - q).C' (degree 5, the T matrix of
//      Sec. 4.3), each coefficient compared with a bound on its FP32
//      rounding error:
//        one sign change, E(0) < 0 < E(1)  -> exactly one minimum inside:
//                                             SEED (the network's job);
//        no sign change                     -> minimum at u = 0 or u = 1;
//        one change, E(0) > 0 > E(1)        -> a maximum inside: the smaller
//                                             end;
//        more changes, or a coefficient within its rounding bound of 0
//                                           -> certified isolation (ISO).
//      A pair whose minimum is at an end is dropped when its FP32 distance
//      there, less its rounding bound, exceeds the query's upper bound (most
//      pairs that pass the box test are of this kind).  Pairs go to one
//      buffer: seeds from the front, the others from the back, so the
//      network reads a dense range.
//   2. the fused MLP (mlp.cu) writes the seed u0 of every SEED pair (without
//      a network: u0 = 1/2).
//   3. one thread per pair: FP32 Newton in the segment's local frame
//      (bracketed by the known sign change for SEED pairs) and a bound on the
//      FP32 distance's rounding error; per-query minimum of the upper bounds
//      by an integer atomicMin on the float bits; then the two FP64 Newton
//      steps (and the FP64 safeguarded iteration when the second step is not
//      below 1e-9) for the pairs whose lower bound does not exceed their
//      query's best upper bound; then the per-query
//      lexicographic minimum over (D, segment) by two more atomicMin passes,
//      the unique winning pair is recorded per query, and one pass over the
//      queries writes every result once (Sec. 4.4.2).
//   4. queries whose pairs did not fit the buffer run through the grid
//      kernel (mixed precision) over a device-side list.
#include "../../include/bspl_mlp.h"
#include "query_common.cuh"
#include "clip.cuh"
#include "tc05.cuh"

namespace bspl {

cudaError_t mlp_seed_pairs(const bspl_mlp* m, const int32_t* pq, const int32_t* ps, const float* qrec,
                           const bspl_segments* segs, int64_t cap, const unsigned long long* n_dev, float* u0,
                           cudaStream_t s);

namespace {

constexpr int kPairsPerQuery = 24;  // buffer capacity per query

struct PairBuf {
    int32_t* pq;              // sorted query position (the query index when collecting)
    int32_t* ps;
    uint8_t* kind;
    float* u;
    float* D32;               // lower bound of the pair's distance (FP32 stage)
    uint8_t* conv;            // 0: FP32 not converged, 1: converged, 2: FP64 must decide among all
                              // minima (both ends for kEnds)
    double* D64;
    double* u64;
    uint8_t* fl;
    int64_t cap;
    unsigned long long* cnt;  // [0] reserved, [1] seeds, [2] others, [3] overflowed queries, [4] finished,
                              // [5] deferred to the FP64 isolation, [6] culling batches taken,
                              // [7] culling candidates reserved
    int32_t* fin;             // buffer slots of the pairs that got the FP64 finish
    int32_t* iso;             // buffer slots of the pairs deferred to the FP64 isolation
    const float* qrec;        // per sorted query: q hi[3], q lo[3], eps, curve (int bits; -1 invalid)
    const int32_t* order;     // sorted position -> query index
    int32_t* over;            // overflowed query indices
    unsigned long long* work; // work-stealing batch counter of the culling launch (zeroed), or NULL
    unsigned* best32;         // per query: FP32 upper bound of the distance (float bits)
    unsigned long long* best64;
    int* bestseg;
    int32_t* cpos;            // culling candidates: sorted query position,
    int32_t* cseg;            //   segment
    float* clb;               //   and squared distance lower bound of its box
    int64_t ccap;
    float* ubq;               // per sorted query: its slacked squared upper bound after culling
    int32_t* wslot;           // per sorted query: buffer slot of the winning pair, or -1
    int32_t* ovf;             // per sorted query: 1 once it is sent to the grid kernel
};


// the cubic C(u) - q in FP32 with a0 - q formed from the high and low FP32
// parts of both (qr: q hi[3], q lo[3]), so no FP64 instruction is needed
__device__ __forceinline__ void local32(const CurveQ& P, int64_t seg, const float* qr, float* c)
{
    const float* r = P.rec32 + (int64_t)BSPL_CREC32 * seg;
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = (r[6 + k] - qr[k]) + (r[18 + k] - qr[3 + k]);
#pragma unroll
    for (int i = 3; i < 12; ++i) c[i] = r[6 + i];
}

// per sorted query: the FP32 parts of q, the FP32 slack and the curve, so
// that the culling kernels run without FP64 instructions (on this GPU one
// FP64 warp instruction occupies its pipe for tens of cycles)
__global__ void k_qrec(const int32_t* __restrict__ qc, const double* __restrict__ q_xyz,
                       const double* __restrict__ diag, int64_t n, int64_t n_q, PairBuf B)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n_q) return;
    float* qrec = const_cast<float*>(B.qrec);
    const int64_t i = B.order[pos];
    B.best32[pos] = 0x7f800000u;
    B.best64[pos] = 0x7ff0000000000000ull;
    B.bestseg[pos] = 0x7fffffff;
    B.wslot[pos] = -1;
    B.ovf[pos] = 0;
    const int c = qc[i];
    float o[8];
    bool bad = c < 0 || c >= n;
    float l1 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x = q_xyz[3 * i + k];
        bad = bad || !isfinite(x);
        o[k] = (float)x;
        o[3 + k] = (float)(x - (double)o[k]);
        l1 += fabsf(o[k]);
    }
    o[6] = bad ? 0.f : 4e-6f * (l1 + (float)diag[c]);
    o[7] = __int_as_float(bad ? -1 : c);
    float4* d = reinterpret_cast<float4*>(qrec + 8 * pos);
    d[0] = make_float4(o[0], o[1], o[2], o[3]);
    d[1] = make_float4(o[4], o[5], o[6], o[7]);
}

constexpr int kCandCap2 = 160; // candidates of a warp batch staged before one global reservation
constexpr int kGrpChunk = 64;  // culling groups staged in shared memory per bulk copy
constexpr int kSurvCap = 128;  // surviving (query, group) entries per warp batch
constexpr uint64_t kCopyWaitNs = 1000000000ull;

// set when a bulk-copy wait gave up (the kernel then reads global memory)
__device__ int g_copy_timeout;

// Culling in two levels.  Level 1 is done for the whole batch of 32 sorted
// queries at once, one lane per query: the curve's group records (box and
// reference point) are staged into shared memory by bulk copies (TMA,
// cp.async.bulk), chunk by chunk, and every lane scans them for its query:
// first the upper bound from the reference points, then the box test; the
// surviving (query, group) pairs go to a per-warp list.  Level 2 is warp-
// cooperative per query over its surviving groups' segments, as in the grid
// kernel; the candidates are filtered against the queries' current bounds,
// staged and written out in bulk for k_classify.
// MINB: blocks per SM the register allocation must allow (1: the compiler's
// choice; 6 or 8 blocks of 4 warps, the latter with a few spilled registers)
template <int MINB>
__global__ void __launch_bounds__(kWarps * 32, MINB) k_cull_cands(CurveQ P, PairBuf B)
{
    // at 8 blocks per SM the shared memory holds one segment-record buffer
    // per warp (the other warps of the SM hide the copy); below, two
    constexpr bool kDouble = MINB < 8;
    __shared__ int s_seg[kWarps][kCandCap2];
    __shared__ float s_lb[kWarps][kCandCap2];
    __shared__ uint8_t s_cslot[kWarps][kCandCap2];
    // level 1 stages group records here; level 2 reuses it as one of the two
    // buffers of segment records (BSPL_GROUP x BSPL_CREC32 floats = the same 3 KB)
    __shared__ __align__(128) float s_grp[kWarps][kGrpChunk * BSPL_GREC32];
    __shared__ __align__(128) float s_seg2[kWarps][kDouble ? BSPL_GROUP * BSPL_CREC32 : 4];
    __shared__ int s_sv[kWarps][kSurvCap];       // surviving groups of the batch, in order
    __shared__ unsigned s_svm[kWarps][kSurvCap]; // the query slots that kept each
    __shared__ __align__(8) uint64_t s_bar[kWarps][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* cseg = s_seg[wid];
    float* clb = s_lb[wid];
    uint8_t* ctslot = s_cslot[wid];
    float* grs = s_grp[wid];
    uint64_t* bar = &s_bar[wid][0];
    const float* rec = P.rec32;
    const float* grp = P.grp32;
    constexpr int RW = BSPL_CREC32, GW = BSPL_GREC32;
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(bar + 1, 1);
        tc::fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0, phase1 = 0;  // parities of the two barriers (they carry over between batches)
    // persistent: each warp takes batches of 32 sorted queries until none is left
    const int64_t nbatch = (P.n_q + kQPW - 1) / kQPW;
    int round = 0;
    for (int64_t batch = next_batch(B.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round); batch < nbatch;
         batch = next_batch(B.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round)) {
    const int64_t qbase = batch * kQPW;
    const int nslots = (int)min((int64_t)kQPW, P.n_q - qbase);
    unsigned long long n_grp = 0, n_seg = 0;
    unsigned over_mask = 0;  // query slots with candidates that did not fit the buffer

    // this lane's query (lane = slot)
    float qx = 0.f, qy = 0.f, qz = 0.f, eps = 0.f;
    int myc = -1;
    if (lane < nslots) {
        const int64_t pos = qbase + lane;
        const float4 qa = *reinterpret_cast<const float4*>(B.qrec + 8 * pos);
        const float4 qb = *reinterpret_cast<const float4*>(B.qrec + 8 * pos + 4);
        qx = qa.x;
        qy = qa.y;
        qz = qa.z;
        eps = qb.z;
        myc = __float_as_int(qb.w);
    }

    // stage groups [g, g + n) of the group table; returns where to read them
    auto stage = [&](int64_t g, int n) -> const float* {
        __syncwarp();
        if (lane == 0) {
            tc::fence_async_smem();  // earlier reads of the buffer come first
            tc::bulk_load(grs, grp + (int64_t)GW * g, (uint32_t)(n * GW * sizeof(float)), bar);
        }
        const bool ok = tc::mbar_wait(bar, phase, kCopyWaitNs);
        phase ^= 1;
        if (!ok && lane == 0) atomicExch(&g_copy_timeout, 1);
        return __all_sync(kFull, ok) ? grs : grp + (int64_t)GW * g;
    };

    // ---- level 1: runs of consecutive slots on the same curve
    int nsv = 0;
    unsigned sv_over = 0;  // slots whose surviving groups did not fit the list
    bool done = !(lane < nslots && myc >= 0);
    float ub = INFINITY;
    for (;;) {
        const unsigned pend = __ballot_sync(kFull, !done);
        if (!pend) break;
        const int c = __shfl_sync(kFull, myc, __ffs(pend) - 1);
        const bool in_run = !done && myc == c;
        const int64_t g0 = P.grp_off[c], G = P.grp_off[c + 1] - g0;
        const float* src = nullptr;
        for (int64_t cg = 0; cg < G; cg += kGrpChunk) {
            const int n = (int)min((int64_t)kGrpChunk, G - cg);
            src = stage(g0 + cg, n);
            if (in_run)
                for (int k = 0; k < n; ++k) ub = fminf(ub, pt_d2(src + GW * k + 6, qx, qy, qz));
        }
        const float ubs = slacked(ub, eps);
        for (int64_t cg = 0; cg < G; cg += kGrpChunk) {
            const int n = (int)min((int64_t)kGrpChunk, G - cg);
            if (G > kGrpChunk) src = stage(g0 + cg, n);
            for (int k = 0; k < n; ++k) {
                const float lb = in_run ? box_d2(src + GW * k, qx, qy, qz) : INFINITY;
                // only this run's queries: a lane outside it may hold an
                // infinite bound (not yet scanned), which lb <= ubs would pass
                const bool keep = in_run && lb <= ubs;
                const unsigned m = __ballot_sync(kFull, keep);
                if (!m) continue;
                if (nsv < kSurvCap) {
                    if (lane == 0) {
                        s_sv[wid][nsv] = (int)(g0 + cg + k);
                        s_svm[wid][nsv] = m;
                    }
                    ++nsv;
                } else {
                    sv_over |= m;
                }
            }
        }
        if (in_run) n_grp += (unsigned long long)G;
        done = done || in_run;
    }
    __syncwarp();

    // ---- level 2: every surviving (query, group) entry of the batch, in
    // list order; lanes = the group's 32 segments.  Each query's upper bound
    // lives in its own lane and tightens as its entries are scanned; the
    // candidates of all queries share one staging buffer, which is filtered
    // against the current bounds and written out in bulk when it fills.
    int64_t s0l = 0, s1l = 0, g0l = 0;
    if (lane < nslots && myc >= 0) {
        s0l = P.seg_off[myc];
        s1l = P.seg_off[myc + 1];
        g0l = P.grp_off[myc];
    }
    float ubs_l = slacked(ub, eps);
    int ncand = 0;
    auto flush_cands = [&]() {
        __syncwarp();
        int nk = 0;
        for (int base = 0; base < ncand; base += 32) {
            const int k = base + lane;
            const bool in = k < ncand;
            const int sl = in ? ctslot[k] : 0;
            const float ubk = __shfl_sync(kFull, ubs_l, sl);
            const float lb = in ? clb[k] : 0.f;
            const int seg = in ? cseg[k] : 0;
            const bool keep = in && lb <= ubk;
            const unsigned m = __ballot_sync(kFull, keep);
            __syncwarp();  // every lane has read its entry before the compaction writes
            if (keep) {
                const int j = nk + __popc(m & lt);
                cseg[j] = seg;
                clb[j] = lb;
                ctslot[j] = (uint8_t)sl;
            }
            nk += __popc(m);
        }
        __syncwarp();
        if (nk > 0) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(B.cnt + 7, (unsigned long long)nk);
            base = __shfl_sync(kFull, base, 0);
            unsigned om = 0;
            for (int k = lane; k < nk; k += 32) {
                const int64_t j = (int64_t)base + k;
                if (j < B.ccap) {
                    B.cpos[j] = (int32_t)(qbase + ctslot[k]);
                    B.cseg[j] = cseg[k];
                    B.clb[j] = clb[k];
                } else {
                    om |= 1u << ctslot[k];
                }
            }
            over_mask |= __reduce_or_sync(kFull, om);
        }
        ncand = 0;
        __syncwarp();
    };
    // box lower bounds and start-point upper bound of one segment per lane
    struct Ent {
        float b[6], p[3];
        int64_t s;
        bool valid;
        int sl;
        int nseg;
    };
    auto scan = [&](const Ent& E) {
        const int sl = E.sl;
        const float sx = __shfl_sync(kFull, qx, sl), sy = __shfl_sync(kFull, qy, sl), sz = __shfl_sync(kFull, qz, sl);
        float lbs = INFINITY, ups = INFINITY;
        if (E.valid) {
            lbs = box_d2(E.b, sx, sy, sz);
            ups = pt_d2(E.p, sx, sy, sz);
        }
        if (lane == E.sl) n_seg += (unsigned long long)E.nseg;
        const float m = warp_min_nonneg(ups);
        if (lane == sl && m < ub) {
            ub = m;
            ubs_l = slacked(ub, eps);
        }
        const float ubs = __shfl_sync(kFull, ubs_l, sl);
        const bool keep = E.valid && lbs <= ubs;
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) {
            const int pos = ncand + __popc(km & lt);
            cseg[pos] = (int)E.s;
            clb[pos] = lbs;
            ctslot[pos] = (uint8_t)sl;
        }
        ncand += __popc(km);
        if (ncand > kCandCap2 - 32) flush_cands();
    };
    auto scan_entry = [&](int sl, int64_t g) {
        const int64_t s0 = __shfl_sync(kFull, s0l, sl), s1 = __shfl_sync(kFull, s1l, sl);
        const int64_t g0 = __shfl_sync(kFull, g0l, sl);
        const int64_t ss = s0 + (g - g0) * BSPL_GROUP;
        const int64_t se = min(ss + BSPL_GROUP, s1);
        Ent E;
        E.sl = sl;
        E.s = ss + lane;
        E.nseg = (int)(se - ss);
        E.valid = E.s < se;
        if (E.valid) {
            const float* r = rec + (int64_t)RW * E.s;
#pragma unroll
            for (int k = 0; k < 6; ++k) E.b[k] = r[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) E.p[k] = r[6 + k];
        }
        scan(E);
    };
    // level 2 over the surviving groups, in list order: a group's segment
    // records are bulk-copied into shared memory once (with two buffers the
    // copy of the next group is in flight while this one is scanned), then
    // every query slot that kept the group scans it warp-cooperatively, one
    // segment per lane, reading the records from shared memory.
    if (nsv > 0) {
        float* buf[2] = { s_grp[wid], kDouble ? s_seg2[wid] : s_grp[wid] };
        // segment range of list entry j (the curve of the first query that kept it)
        auto range = [&](int j, int64_t& ss, int& ns) {
            const int g = s_sv[wid][j];
            const int sl = __ffs(s_svm[wid][j]) - 1;
            const int64_t s0 = __shfl_sync(kFull, s0l, sl), s1 = __shfl_sync(kFull, s1l, sl);
            const int64_t g0 = __shfl_sync(kFull, g0l, sl);
            ss = s0 + ((int64_t)g - g0) * BSPL_GROUP;
            ns = (int)min((int64_t)BSPL_GROUP, s1 - ss);
        };
        auto issue = [&](int j, int b) {
            int64_t ss;
            int ns;
            range(j, ss, ns);
            __syncwarp();  // every lane is done with the buffer's previous contents
            if (lane == 0) {
                tc::fence_async_smem();
                tc::bulk_load(buf[b], rec + (int64_t)RW * ss, (uint32_t)(ns * RW * sizeof(float)), bar + b);
            }
        };
        if (kDouble) issue(0, 0);
        for (int j = 0; j < nsv; ++j) {
            const int b = kDouble ? (j & 1) : 0;
            if (!kDouble) issue(j, 0);
            else if (j + 1 < nsv) issue(j + 1, b ^ 1);
            int64_t ss;
            int ns;
            range(j, ss, ns);
            const bool ok = tc::mbar_wait(bar + b, b ? phase1 : phase, kCopyWaitNs);
            if (b) phase1 ^= 1;
            else phase ^= 1;
            if (!ok && lane == 0) atomicExch(&g_copy_timeout, 1);
            const float* src = __all_sync(kFull, ok) ? buf[b] : rec + (int64_t)RW * ss;
            // this lane's segment of the group
            Ent E;
            E.s = ss + lane;
            E.nseg = ns;
            E.valid = lane < ns;
            if (E.valid) {
                const float* r = src + RW * lane;
#pragma unroll
                for (int k = 0; k < 6; ++k) E.b[k] = r[k];
#pragma unroll
                for (int k = 0; k < 3; ++k) E.p[k] = r[6 + k];
            }
            // the slots that kept the group, if its box still passes their bound
            const float* gr = grp + (int64_t)GW * s_sv[wid][j];
            const bool pass = ((s_svm[wid][j] >> lane) & 1u) && box_d2(gr, qx, qy, qz) <= ubs_l;
            for (unsigned m = __ballot_sync(kFull, pass); m; m &= m - 1) {
                E.sl = __ffs(m) - 1;
                scan(E);
            }
            __syncwarp();
        }
    }
    // queries whose surviving groups did not fit the list: scan all groups
    for (unsigned ov = sv_over; ov; ov &= ov - 1) {
        const int sl = __ffs(ov) - 1;
        const int c = __shfl_sync(kFull, myc, sl);
        const float sx = __shfl_sync(kFull, qx, sl), sy = __shfl_sync(kFull, qy, sl), sz = __shfl_sync(kFull, qz, sl);
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];
        for (int64_t gb = g0; gb < g1; gb += 32) {
            const int64_t g = gb + lane;
            const float lbg = g < g1 ? box_d2(grp + (int64_t)GW * g, sx, sy, sz) : INFINITY;
            unsigned m = __ballot_sync(kFull, lbg <= __shfl_sync(kFull, ubs_l, sl));
            while (m) {
                const int jg = __ffs(m) - 1;
                m &= m - 1;
                if (__shfl_sync(kFull, lbg, jg) <= __shfl_sync(kFull, ubs_l, sl)) scan_entry(sl, gb + jg);
            }
        }
    }
    flush_cands();
    if (lane < nslots) {
        const int64_t pos = qbase + lane;
        B.ubq[pos] = ubs_l;
        if (((over_mask >> lane) & 1u) && atomicExch(B.ovf + pos, 1) == 0)
            B.over[atomicAdd(B.cnt + 3, 1ull)] = B.order[pos];
    }
    if (P.counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n_grp += __shfl_xor_sync(kFull, n_grp, o);
            n_seg += __shfl_xor_sync(kFull, n_seg, o);
        }
        if (lane == 0) {
            atomicAdd(P.counters + BSPL_CNT_QUERIES, (unsigned long long)nslots);
            atomicAdd(P.counters + BSPL_CNT_GRP_TESTED, n_grp);
            atomicAdd(P.counters + BSPL_CNT_SEG_TESTED, n_seg);
        }
    }
    __syncwarp();
    }  // batches
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

// Classification of every culling candidate, one thread per candidate (Sec.
// 4.3: the signs of the Bernstein coefficients of E, each against its FP32
// rounding bound), and the emission of the pairs that can hold their
// query's minimum: SEED pairs to the front of the pair buffer, the others to
// the back.  A candidate whose box bound exceeds its query's final upper
// bound is dropped, and so is a pair whose minimum is at an end when its
// FP32 distance there less its rounding bound exceeds that bound.  A block
// takes kClsRounds x 256 candidates at a time and reserves its slots in the
// buffer once; when they do not fit, the queries concerned go to the grid
// kernel.  SEEDS_ONLY: only SEED pairs, written with the query index (the
// network's training pairs).
constexpr int kClsRounds = 4;

template <bool SEEDS_ONLY>
__global__ void __launch_bounds__(256) k_classify(CurveQ P, PairBuf B)
{
    __shared__ int s_ns[kClsRounds][8], s_no[kClsRounds][8];
    __shared__ unsigned long long s_bs, s_bo;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nc = min((int64_t)B.cnt[7], B.ccap);
    unsigned long long n_cls = 0, n_emit = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * 256 * kClsRounds; c0 < nc;
         c0 += (int64_t)gridDim.x * 256 * kClsRounds) {
        int pos[kClsRounds], seg[kClsRounds];
        uint8_t kind[kClsRounds];
        unsigned ms[kClsRounds], mo[kClsRounds];
#pragma unroll
        for (int r = 0; r < kClsRounds; ++r) {
            const int64_t j = c0 + r * 256 + threadIdx.x;
            bool keep = false;
            pos[r] = 0;
            seg[r] = 0;
            kind[r] = kIso;
            if (j < nc) {
                pos[r] = B.cpos[j];
                seg[r] = B.cseg[j];
                const float ubk = B.ubq[pos[r]];
                if (B.clb[j] <= ubk) {
                    float cl[12];
                    local32(P, seg[r], B.qrec + 8 * (int64_t)pos[r], cl);
                    kind[r] = classify(cl);
                    ++n_cls;
                    keep = !SEEDS_ONLY || kind[r] == kSeed;
                    if (!SEEDS_ONLY && (kind[r] == kEnd0 || kind[r] == kEnd1 || kind[r] == kEnds)) {
                        // the segment's minimum is at an end: its FP32
                        // distance there less the rounding bound of the FP32
                        // stage is a lower bound of the pair's distance
                        float l1 = 0.f, d0 = 0.f, d1 = 0.f;
#pragma unroll
                        for (int k = 0; k < 12; ++k) l1 += fabsf(cl[k]);
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float e = ((cl[9 + k] + cl[6 + k]) + cl[3 + k]) + cl[k];
                            d0 += cl[k] * cl[k];
                            d1 += e * e;
                        }
                        const float dm = kind[r] == kEnd0 ? d0 : (kind[r] == kEnd1 ? d1 : fminf(d0, d1));
                        keep = sqrtf(dm) - 1e-6f * l1 <= sqrtf(ubk);
                    }
                }
            }
            ms[r] = __ballot_sync(kFull, keep && kind[r] == kSeed);
            mo[r] = __ballot_sync(kFull, keep && kind[r] != kSeed);
            if (lane == 0) {
                s_ns[r][wid] = __popc(ms[r]);
                s_no[r][wid] = __popc(mo[r]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // exclusive prefix over (round, warp), then one reservation
            int ns = 0, no = 0;
            for (int r = 0; r < kClsRounds; ++r)
                for (int w = 0; w < 8; ++w) {
                    const int a = s_ns[r][w], b = s_no[r][w];
                    s_ns[r][w] = ns;
                    s_no[r][w] = no;
                    ns += a;
                    no += b;
                }
            int ok = 1;
            unsigned long long bs = 0, bo = 0;
            if (ns + no > 0) {
                const unsigned long long tot = atomicAdd(B.cnt, (unsigned long long)(ns + no));
                ok = tot + ns + no <= (unsigned long long)B.cap;
                if (ok) {
                    bs = ns ? atomicAdd(B.cnt + 1, (unsigned long long)ns) : 0;
                    bo = no ? atomicAdd(B.cnt + 2, (unsigned long long)no) : 0;
                }
            }
            s_ok = ok;
            s_bs = bs;
            s_bo = bo;
        }
        __syncthreads();
        const bool ok = s_ok;
#pragma unroll
        for (int r = 0; r < kClsRounds; ++r) {
            const bool sd = (ms[r] >> lane) & 1u, ot = (mo[r] >> lane) & 1u;
            if (!(sd || ot)) continue;
            if (!ok) {
                if (!SEEDS_ONLY && atomicExch(B.ovf + pos[r], 1) == 0)
                    B.over[atomicAdd(B.cnt + 3, 1ull)] = B.order[pos[r]];
                continue;
            }
            ++n_emit;
            if (sd) {
                const int64_t idx = (int64_t)s_bs + s_ns[r][wid] + __popc(ms[r] & lt);
                B.pq[idx] = SEEDS_ONLY ? B.order[pos[r]] : pos[r];
                B.ps[idx] = seg[r];
                if (B.kind) B.kind[idx] = kSeed;
            } else {
                const int64_t idx = B.cap - 1 - ((int64_t)s_bo + s_no[r][wid] + __popc(mo[r] & lt));
                B.pq[idx] = pos[r];
                B.ps[idx] = seg[r];
                B.kind[idx] = kind[r];
            }
        }
        __syncthreads();
    }
    if (!SEEDS_ONLY && P.counters) {
        add_counter(P.counters, BSPL_CNT_CANDIDATES, n_emit);
        add_counter(P.counters, BSPL_CNT_CLASSIFIED, n_cls);
    }
}

// (3a) FP32 solve of every pair, per-query FP32 minimum.  CLIP: the pairs
// with a minimum inside (one certified sign change, or more) are solved by
// the paper's search (monotone split by the roots of E', elimination,
// Bezier clipping; clip.cuh) and then by the FP32 Newton steps; a seeded
// pair on which the search does not find exactly one interior minimum is
// left for the FP64 stage to decide.
template <bool CLIP>
__global__ void k_pairs_fp32(CurveQ P, PairBuf B, int have_seed)
{
    const int64_t ns = (int64_t)B.cnt[1], no = (int64_t)B.cnt[2], np = ns + no;
    unsigned it32 = 0, n_iso = 0;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < np; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        if (j < np) {
            const int64_t i = pair_slot(B, j, ns);
            const int64_t pos = B.pq[i], seg = B.ps[i];
            const uint8_t kind = j < ns ? kSeed : B.kind[i];
            float c[12];
            local32(P, seg, B.qrec + 8 * pos, c);
            float u, E, Ep;
            bool conv = true;
            float l1 = 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) l1 += fabsf(c[k]);
            const float del = 1e-6f * l1;
            // ambiguous: the FP32 stage cannot tell which candidate of the
            // pair is the minimum (the FP64 stage then decides among all)
            bool amb = false, unsure = false;
            if (CLIP && kind != kEnd0 && kind != kEnd1 && kind != kEnds) {
                if (kind != kSeed) ++n_iso;
                float b[6], ba[6], second[3];
                bern_E32(c, b, ba);
                ClipOut co;
                u = clip_min<float>(c, 1e-5f * ba[5], 12, second, co);
                unsure = co.unsure || kind == kIsoU || (kind == kSeed && co.n_min != 1);
                conv = newton_min<float>(c, 0.f, 0.f, 0.f, u, 1.f / 64.f, P.fp32_steps, 1e-7f, it32);
                const float dd = sqrtf(eval_E<float>(c, 0.f, 0.f, 0.f, u, E, Ep));
                amb = unsure || sqrtf(second[0]) - dd <= 2.f * del;
            } else if (kind == kSeed) {
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
                amb = fabsf(sqrtf(D1) - sqrtf(D0)) <= 2.f * del;
            } else {
                ++n_iso;
                // isolation with the coefficients' rounding scale: an interval
                // whose sign pattern is not certain makes the pair uncertain
                float b[6], bt[6], second[3];
                bern_E32(c, b, bt);
#pragma unroll
                for (int k = 0; k < 6; ++k) bt[k] *= 1e-5f;  // the classification's rounding bounds
                unsure = kind == kIsoU;
                u = isolate_min<float>(c, 0.f, 0.f, 0.f, 1e-7f, P.fp32_steps * 4, second, bt, &unsure);
                conv = newton_min<float>(c, 0.f, 0.f, 0.f, u, 1.f / 64.f, P.fp32_steps, 1e-7f, it32);
                const float dd = sqrtf(eval_E<float>(c, 0.f, 0.f, 0.f, u, E, Ep));
                amb = unsure || sqrtf(second[0]) - dd <= 2.f * del;
            }
            // FP32 distance and a bound on its error (coefficient rounding
            // and Horner evaluation in the local frame, |u| <= 1)
            const float d = sqrtf(eval_E<float>(c, 0.f, 0.f, 0.f, u, E, Ep));
            B.u[i] = u;
            // lower bound of the pair's distance; an uncertain isolation may
            // have missed the segment's minimum, and an unconverged iterate
            // is not at one: then the distance to the box of the Bezier
            // control points (convex hull) bounds it
            float lbd = d;
            if (unsure || !conv) {
                float s2 = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float p0 = c[k], p1 = c[k] + c[3 + k] * (1.f / 3.f),
                                p2 = c[k] + (2.f * c[3 + k] + c[6 + k]) * (1.f / 3.f),
                                p3 = c[k] + c[3 + k] + c[6 + k] + c[9 + k];
                    const float lo = fminf(fminf(p0, p1), fminf(p2, p3)), hi = fmaxf(fmaxf(p0, p1), fmaxf(p2, p3));
                    const float g = fmaxf(fmaxf(lo, -hi), 0.f);  // the query is the origin of the local frame
                    s2 += g * g;
                }
                lbd = sqrtf(s2);
            }
            B.D32[i] = lbd - del;
            B.conv[i] = amb ? 2 : (conv ? 1 : 0);
            atomicMin(B.best32 + pos, __float_as_uint(d + del));
        }
    }
    if (P.counters) {
        add_counter(P.counters, BSPL_CNT_NEWTON32_ITERS, it32);
        add_counter(P.counters, BSPL_CNT_ISO_PAIRS, n_iso);
    }
}

// (3b) FP64 finish of the pairs whose FP32 lower bound does not exceed their
// query's best upper bound.  A block first lists the pairs of its chunk that
// need the finish, then works through the list with all its threads, so the
// FP64 instructions run in full warps (on this GPU the FP64 pipe is the
// scarce one and a warp with one active lane costs as much as a full one).
constexpr int kFinChunk = 1024;

__global__ void __launch_bounds__(256, 3) k_pairs_fp64(CurveQ P, PairBuf B)
{
    __shared__ int s_list[kFinChunk];
    __shared__ int s_n;
    __shared__ unsigned long long s_base;
    const int64_t ns = (int64_t)B.cnt[1], no = (int64_t)B.cnt[2], np = ns + no;
    unsigned it64 = 0, nfin = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kFinChunk; c0 < np; c0 += (int64_t)gridDim.x * kFinChunk) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < kFinChunk; k += blockDim.x) {
            const int64_t j = c0 + k;
            if (j >= np) break;
            const int64_t i = pair_slot(B, j, ns);
            if (B.conv[i] && B.D32[i] > __uint_as_float(B.best32[B.pq[i]])) B.D64[i] = INFINITY;  // pq: position
            else s_list[atomicAdd(&s_n, 1)] = k;
        }
        __syncthreads();
        const int nt = s_n;
        if (threadIdx.x == 0 && nt > 0) s_base = atomicAdd(B.cnt + 4, (unsigned long long)nt);
        __syncthreads();
        for (int k = threadIdx.x; k < nt; k += blockDim.x) {
            const int64_t j = c0 + s_list[k];
            const int64_t i = pair_slot(B, j, ns);
            B.fin[s_base + k] = (int32_t)i;
            const int64_t pos = B.pq[i], seg = B.ps[i];
            const double* q = P.q_xyz + 3 * (int64_t)B.order[pos];
            ++nfin;
            const uint8_t kind = j < ns ? kSeed : B.kind[i];
            const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * seg + 6;
            double c64[12];
#pragma unroll
            for (int m = 0; m < 12; ++m) c64[m] = a64[m];
            double u = (double)B.u[i], last = 0.0, D = 0.0, E, Ep;
            bool ok = true;
            if (B.conv[i] == 2 && kind == kEnds) {
                // both ends in FP64 (ties: u = 0)
                const double D0 = eval_E(c64, q[0], q[1], q[2], 0.0, E, Ep);
                const double D1 = eval_E(c64, q[0], q[1], q[2], 1.0, E, Ep);
                u = D1 < D0 ? 1.0 : 0.0;
                D = D1 < D0 ? D1 : D0;
            } else {
                // an undecided pair is classified again from E's Bernstein
                // coefficients in FP64: no sign change, or one from + to -,
                // puts the minimum at an end; one from - to + is a single
                // interior minimum (the FP64 steps from the FP32 iterate);
                // more go to the certified FP64 isolation
                int v64 = 1;
                bool at_end = false;
                if (B.conv[i] == 2) {
                    double b64[6];
                    int sf, sl;
                    v64 = bernstein_E<double>(c64, q[0], q[1], q[2], b64);
                    end_signs6(b64, sf, sl);
                    at_end = v64 == 0 || (v64 == 1 && sf > 0);
                }
                if (at_end) {
                    const double D0 = eval_E(c64, q[0], q[1], q[2], 0.0, E, Ep);
                    const double D1 = eval_E(c64, q[0], q[1], q[2], 1.0, E, Ep);
                    u = D1 < D0 ? 1.0 : 0.0;
                    D = D1 < D0 ? D1 : D0;
                    ok = true;
                } else if (v64 == 1) {
                    D = finish64(c64, P.rec32 + (int64_t)BSPL_CREC32 * seg + 9, q, u, last, it64);
                    ok = last <= 1e-9;
                } else {
                    ok = false;
                }
                if (!ok) {
                    // to the FP64 isolation, run over a compact list in full warps
                    B.iso[atomicAdd(B.cnt + 5, 1ull)] = (int32_t)i;
                    continue;
                }
            }
            const uint8_t fl = BSPL_Q_CONVERGED;
            B.D64[i] = D;
            B.u64[i] = u;
            B.fl[i] = fl;
            atomicMin(B.best64 + pos, (unsigned long long)__double_as_longlong(D));
        }
        __syncthreads();
    }
    if (P.counters) {
        add_counter(P.counters, BSPL_CNT_NEWTON64_ITERS, it64);
        add_counter(P.counters, BSPL_CNT_NEWTON, nfin);
    }
}

// (3b') the FP64 fallback: certified isolation of every minimum of the
// segment (Bernstein sign variations of E in FP64), then the safeguarded
// iteration from the best one.  Taken by the pairs whose two FP64 steps did
// not converge and by those the FP32 stage could not decide (an uncertain
// sign pattern, or two candidates within the FP32 error bound of each other:
// e.g. two minima of a near-cusp a few hundredths apart).  A separate pass
// over a compact list, so the long FP64 iteration runs in full warps.
__global__ void k_pairs_iso64(CurveQ P, PairBuf B)
{
    const int64_t n = (int64_t)B.cnt[5];
    unsigned it64 = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = B.iso[j];
        const int64_t pos = B.pq[i], seg = B.ps[i];
        const double* q = P.q_xyz + 3 * (int64_t)B.order[pos];
        const double* a64 = P.rec64 + (int64_t)BSPL_CREC64 * seg + 6;
        double c64[12];
#pragma unroll
        for (int m = 0; m < 12; ++m) c64[m] = a64[m];
        double u = isolate_min<double>(c64, q[0], q[1], q[2], 1e-15, P.newton_max);
        const bool ok = newton_min<double>(c64, q[0], q[1], q[2], u, 1.0 / 64, P.newton_max, 1e-15, it64);
        double E, Ep;
        const double D = eval_E(c64, q[0], q[1], q[2], u, E, Ep);
        B.D64[i] = D;
        B.u64[i] = u;
        B.fl[i] = BSPL_Q_FALLBACK | (ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV);
        atomicMin(B.best64 + pos, (unsigned long long)__double_as_longlong(D));
    }
    if (P.counters) add_counter(P.counters, BSPL_CNT_NEWTON64_ITERS, it64);
}

// (3c) smallest segment among the pairs at the query's best FP64 distance
__global__ void k_pairs_argseg(CurveQ P, PairBuf B)
{
    const int64_t nf = (int64_t)B.cnt[4];  // only finished pairs can hold a query's minimum
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = B.fin[j];
        const int64_t pos = B.pq[i];
        if ((unsigned long long)__double_as_longlong(B.D64[i]) == B.best64[pos]) atomicMin(B.bestseg + pos, B.ps[i]);
    }
}

// (3d) the winning pair of each query: the unique finished pair at its
// best (D, segment)
__global__ void k_pairs_win(CurveQ P, PairBuf B)
{
    const int64_t nf = (int64_t)B.cnt[4];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = B.fin[j];
        const int64_t pos = B.pq[i];
        if ((unsigned long long)__double_as_longlong(B.D64[i]) == B.best64[pos] && B.ps[i] == B.bestseg[pos])
            B.wslot[pos] = (int32_t)i;
    }
}

// (3e) every query's result, once, in sorted order: the winning pair's
// parameter mapped to the original one (Sec. 4.4.2), its distance and
// flags.  An invalid query gets NaN and INVALID; a valid one without a
// winner (none is expected: the pair holding the minimum is never dropped)
// NaN and NONCONV; the queries sent to the grid kernel are left to it.
// (Writing in the caller's order instead, through the inverse of the sort,
// turns these scattered writes into scattered reads of the per-query data
// and measured slower.)
__global__ void k_write_results(CurveQ P, PairBuf B)
{
    unsigned fb = 0, nc = 0;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < P.n_q; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = j0 + threadIdx.x;
        if (pos >= P.n_q || B.ovf[pos]) continue;
        const int64_t qi = B.order[pos];
        const int c = __float_as_int(B.qrec[8 * pos + 7]);
        double t = __longlong_as_double(0x7ff8000000000000LL), d = t;
        unsigned char fl = BSPL_Q_INVALID;
        if (c >= 0) {
            const int32_t i = B.wslot[pos];
            fl = BSPL_Q_NONCONV;
            if (i >= 0) {
                const int seg = B.ps[i];
                const double u = B.u64[i];
                const double t0 = P.prange[2 * seg], t1 = P.prange[2 * seg + 1];
                t = u <= 0.0 ? t0 : (u >= 1.0 ? t1 : t0 + u * (t1 - t0));
                d = sqrt(B.D64[i]);
                fl = B.fl[i];
                if ((seg == P.seg_off[c] && u <= 0.0) || (seg == P.seg_off[c + 1] - 1 && u >= 1.0))
                    fl |= BSPL_Q_AT_END;
                if (P.invert && d > 1e-9 * P.diag[c]) fl |= BSPL_Q_OFF_CURVE;
            }
            fb += (fl & BSPL_Q_FALLBACK) ? 1 : 0;
            nc += (fl & BSPL_Q_NONCONV) ? 1 : 0;
        }
        P.t[qi] = t;
        P.dist[qi] = d;
        P.status[qi] = fl;
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
    B.cnt = cv.take<unsigned long long>(8);
    B.fin = cv.take<int32_t>((size_t)cap);
    B.iso = cv.take<int32_t>((size_t)cap);
    B.qrec = cv.take<float>((size_t)n_q * 8);
    B.ccap = cap;
    B.cpos = cv.take<int32_t>((size_t)cap);
    B.cseg = cv.take<int32_t>((size_t)cap);
    B.clb = cv.take<float>((size_t)cap);
    B.ubq = cv.take<float>((size_t)n_q);
    B.wslot = cv.take<int32_t>((size_t)n_q);
    B.ovf = cv.take<int32_t>((size_t)n_q);
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
    if (!segs_ok(segs) || n_q < 0 || pair_cap(n_q) > 0x7fffffffLL) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    if (!q_curve || !q_xyz || !t || !dist || !status) return BSPL_EINVAL;
    const bspl_mlp* mlp = o->prec == BSPL_CLIP_MIXED ? nullptr : (const bspl_mlp*)o->mlp;
    if (mlp && (!mlp->params || !mlp->wbf16 || mlp->kind != BSPL_MLP_CURVE)) return BSPL_EINVAL;
    if (o->occupancy < 0 || o->occupancy > 2) return BSPL_EINVAL;
    if (o->pairs_per_query < 0 || o->pairs_per_query > kPairsPerQuery) return BSPL_EINVAL;
    PairBuf B{};
    void* sw = nullptr;
    size_t sb = 0;
    if (!carve_learned(ws, ws_bytes, segs->n, n_q, B, &sw, &sb, nullptr)) return BSPL_EINVAL;
    if (o->pairs_per_query > 0) B.cap = o->pairs_per_query * n_q;  // the rest of the buffer stays unused
    CurveQ P = make_params(segs, n_q, q_curve, q_xyz, *o, invert, t, dist, status);
    const cudaEvent_t* ev = (const cudaEvent_t*)o->stage_events;
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], s);
    };
    mark(0);
    int32_t* order = nullptr;
    if (sort_by_spline(q_curve, n_q, segs->n, segs->spline_rank, sw, sb, &order, nullptr, s) != cudaSuccess)
        return BSPL_ECUDA;
    P.order = order;
    B.order = order;
    k_qrec<<<ceil_div(n_q, 256), 256, 0, s>>>(q_curve, q_xyz, segs->diag, segs->n, n_q, B);
    if (cudaMemsetAsync(B.cnt, 0, 8 * sizeof(unsigned long long), s) != cudaSuccess) return BSPL_ECUDA;
    mark(1);
    const int64_t blocks = (n_q + kQPW * kWarps - 1) / (kQPW * kWarps);
    B.work = B.cnt + 6;  // zeroed with the other counters
    if (o->occupancy >= 2)
        k_cull_cands<8><<<persistent_blocks(k_cull_cands<8>, kWarps * 32, 0, blocks), kWarps * 32, 0, s>>>(P, B);
    else if (o->occupancy == 1)
        k_cull_cands<6><<<persistent_blocks(k_cull_cands<6>, kWarps * 32, 0, blocks), kWarps * 32, 0, s>>>(P, B);
    else
        k_cull_cands<1><<<persistent_blocks(k_cull_cands<1>, kWarps * 32, 0, blocks), kWarps * 32, 0, s>>>(P, B);
    mark(2);
    const int grid = pair_grid();
    k_classify<false><<<grid, 256, 0, s>>>(P, B);
    mark(3);
    if (mlp && mlp_seed_pairs(mlp, B.pq, B.ps, B.qrec, segs, B.cap, B.cnt + 1, B.u, s) != cudaSuccess)
        return BSPL_ECUDA;
    mark(4);
    if (o->prec == BSPL_CLIP_MIXED) k_pairs_fp32<true><<<grid, 256, 0, s>>>(P, B, 0);
    else k_pairs_fp32<false><<<grid, 256, 0, s>>>(P, B, mlp ? 1 : 0);
    mark(5);
    k_pairs_fp64<<<grid, 256, 0, s>>>(P, B);
    k_pairs_iso64<<<grid, 128, 0, s>>>(P, B);
    mark(6);
    k_pairs_argseg<<<grid, 256, 0, s>>>(P, B);
    k_pairs_win<<<grid, 256, 0, s>>>(P, B);
    k_write_results<<<grid, 256, 0, s>>>(P, B);
    mark(7);
    // queries whose pairs did not fit: the grid kernel over the device-side list
    CurveQ F = P;
    F.order = B.over;
    F.n_q_dev = reinterpret_cast<const int64_t*>(B.cnt + 3);
    F.counters = nullptr;
    launch_mixed_curves(F, o->occupancy, s);
    mark(8);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl

using namespace bspl;

extern "C" bspl_status bspl_mlp_collect_pairs(const bspl_segments* segs, int64_t n_q, const int32_t* q_curve,
                                              const double* q_xyz, int64_t cap, int32_t* pair_q, int32_t* pair_seg,
                                              int64_t* n_pairs, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    if (!segs_ok(segs) || n_q < 0 || n_q > 0x7fffffffLL || cap < 0 || !n_pairs) return BSPL_EINVAL;
    if (n_q > 0 && (!q_curve || !q_xyz || (cap > 0 && (!pair_q || !pair_seg)))) return BSPL_EINVAL;
    PairBuf B{};
    void* sw = nullptr;
    size_t sb = 0;
    if (!carve_learned(ws, ws_bytes, segs->n, n_q, B, &sw, &sb, nullptr)) return BSPL_EINVAL;
    if (cudaMemsetAsync(B.cnt, 0, 8 * sizeof(unsigned long long), stream) != cudaSuccess) return BSPL_ECUDA;
    if (n_q > 0) {
        bspl_options o{};
        CurveQ P = make_params(segs, n_q, q_curve, q_xyz, o, 0, nullptr, nullptr, nullptr);
        P.counters = nullptr;
        int32_t* order = nullptr;
        if (sort_by_spline(q_curve, n_q, segs->n, segs->spline_rank, sw, sb, &order, nullptr, stream) !=
            cudaSuccess)
            return BSPL_ECUDA;
        P.order = order;
        B.order = order;
        k_qrec<<<ceil_div(n_q, 256), 256, 0, stream>>>(q_curve, q_xyz, segs->diag, segs->n, n_q, B);
        PairBuf C = B;
        C.pq = pair_q;
        C.ps = pair_seg;
        C.kind = nullptr;
        C.cap = cap;
        const int64_t blocks = (n_q + kQPW * kWarps - 1) / (kQPW * kWarps);
        C.work = B.cnt + 6;  // zeroed above
        k_cull_cands<1><<<persistent_blocks(k_cull_cands<1>, kWarps * 32, 0, blocks), kWarps * 32, 0, stream>>>(P, C);
        k_classify<true><<<pair_grid(), 256, 0, stream>>>(P, C);
    }
    if (cudaMemcpyAsync(n_pairs, B.cnt + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(n_pairs + 1, B.cnt, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return BSPL_ECUDA;
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}
