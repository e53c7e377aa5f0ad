// Batched point projection / inversion on decomposed surfaces.
//
// Same organisation as the curve kernel: queries grouped by surface, one warp
// per batch of 32 queries, warp-cooperative culling of patch groups and
// patches, a GU x GV sample grid on each surviving bicubic patch (one or two
// patches per warp step) with basins detected through shuffles against the
// four grid neighbours, and a pooled per-lane Newton phase.
//
// The decomposition of a surface may be coarser than the final accuracy: the
// culling boxes enclose the ORIGINAL piece of every patch, the upper bound
// from sampled bicubic points is widened by the certified deviation
// tol x diag, and the last Newton steps run on the ORIGINAL span-pair patch
// (power basis of degree <= 7 per direction), so the reported (u, v) and
// distance are those of the original surface.
//
// Newton on D(u,v) = |S(u,v) - q|^2 (the 2-D analogue of Eqs. Dt, Et, E't):
// gradient g = (d.S_u, d.S_v), Hessian H = [S_u.S_u + d.S_uu, S_u.S_v + d.S_uv;
// ., S_v.S_v + d.S_vv] with d = S - q, on the box [0,1]^2 with an active set
// (a coordinate on a bound whose gradient points outward is held) and a
// halving safeguard on D.
#include <math.h>

#include "bspl_internal.cuh"

namespace bspl {

cudaError_t sort_by_spline(const int32_t* qc, int64_t n_q, int64_t n, void* ws, size_t ws_bytes, int32_t** order,
                           cudaStream_t s);

namespace {

constexpr int kQPW = 32;
constexpr int kCandCap = 96;
constexpr int kPoolCap = 128;
constexpr int kWarps = 4;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kSN = 8;  // span-pair net stride (degree <= 7)

struct SurfQ {
    const int64_t* seg_off;
    const int64_t* grp_off;
    const double* rec64;
    const float* rec32;
    const double* grp64;
    const float* grp32;
    const double* prange;
    const double* patch_box;
    const int64_t* patch_span;
    const double* span_net;
    const float* span_net32;
    const double* diag;
    double tol_rel;
    int64_t n, n_q;
    const int32_t* q_surf;
    const double* q_xyz;
    const int32_t* order;
    double* uv;
    double* dist;
    uint8_t* status;
    int invert;
    int newton_max;
    int fp32_steps;
    unsigned long long* counters;
};

template <class R>
struct STab;
template <>
struct STab<double> {
    static __device__ const double* rec(const SurfQ& P) { return P.rec64; }
    static __device__ const double* grp(const SurfQ& P) { return P.grp64; }
    static constexpr int RW = BSPL_SREC64, GW = BSPL_GREC64;
};
template <>
struct STab<float> {
    static __device__ const float* rec(const SurfQ& P) { return P.rec32; }
    static __device__ const float* grp(const SurfQ& P) { return P.grp32; }
    static constexpr int RW = BSPL_SREC32, GW = BSPL_GREC32;
};

template <class R>
__device__ __forceinline__ R warp_min(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <class R>
__device__ __forceinline__ R box_d2(const R* b, R qx, R qy, R qz)
{
    R dx = fmax(fmax(b[0] - qx, qx - b[3]), R(0));
    R dy = fmax(fmax(b[1] - qy, qy - b[4]), R(0));
    R dz = fmax(fmax(b[2] - qz, qz - b[5]), R(0));
    return dx * dx + dy * dy + dz * dz;
}

template <class R>
__device__ __forceinline__ R pt_d2(const R* p, R qx, R qy, R qz)
{
    R dx = p[0] - qx, dy = p[1] - qy, dz = p[2] - qz;
    return dx * dx + dy * dy + dz * dz;
}

template <class R>
__device__ __forceinline__ R slacked(R ub, R eps)
{
    R s = sqrt(ub) + eps;
    return s * s;
}

// value and partials up to order 2 of sum_{i<=du, j<=dv} a[i][j] u^i v^j
// (coefficient (i,j) of coordinate c at a[(i*stride + j)*3 + c])
template <class R>
struct SD {
    R S[3], Su[3], Sv[3], Suu[3], Suv[3], Svv[3];
};

template <class R>
__device__ __forceinline__ void eval_patch(const R* a, int du, int dv, int stride, R u, R v, SD<R>& o)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R s = 0, su = 0, sv = 0, suu = 0, suv = 0, svv = 0;
        for (int i = du; i >= 0; --i) {
            // row polynomial in v and its first two derivatives
            R p = 0, p1 = 0, p2 = 0;
            for (int j = dv; j >= 0; --j) {
                R coef = a[(i * stride + j) * 3 + c];
                p2 = p2 * v + R(2) * p1;
                p1 = p1 * v + p;
                p = p * v + coef;
            }
            // Horner in u with derivatives
            suu = suu * u + R(2) * su;
            suv = suv * u + sv;
            su = su * u + s;
            s = s * u + p;
            svv = svv * u + p2;
            sv = sv * u + p1;
        }
        // sv above accumulated d/dv rows; suv accumulated d/du of sv
        o.S[c] = s;
        o.Su[c] = su;
        o.Sv[c] = sv;
        o.Suu[c] = suu;
        o.Suv[c] = suv;
        o.Svv[c] = svv;
    }
}

// squared distance, gradient (halved), Hessian (halved) and the Gauss-Newton
// matrix J^T J of D at one point
template <class R>
struct GH {
    R gu, gv, huu, huv, hvv, juu, juv, jvv;
};

template <class R>
__device__ __forceinline__ R grad_hess(const SD<R>& o, R qx, R qy, R qz, GH<R>& h)
{
    R d[3] = { o.S[0] - qx, o.S[1] - qy, o.S[2] - qz };
    R D = 0;
    h.gu = h.gv = h.huu = h.huv = h.hvv = h.juu = h.juv = h.jvv = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        D += d[c] * d[c];
        h.gu += d[c] * o.Su[c];
        h.gv += d[c] * o.Sv[c];
        h.juu += o.Su[c] * o.Su[c];
        h.juv += o.Su[c] * o.Sv[c];
        h.jvv += o.Sv[c] * o.Sv[c];
        h.huu += d[c] * o.Suu[c];
        h.huv += d[c] * o.Suv[c];
        h.hvv += d[c] * o.Svv[c];
    }
    h.huu += h.juu;
    h.huv += h.juv;
    h.hvv += h.jvv;
    return D;
}

// projected Newton with active set and halving safeguard on [0,1]^2: the
// Newton step where the Hessian is positive definite, the Gauss-Newton step
// (J^T J, positive definite on a regular surface) elsewhere, so the step
// does not depend on how the parameters are scaled.  A coordinate on a bound
// whose gradient points outward is held.  Returns true when converged (step
// below tol, KKT point on the bounds, or no descent left at this precision).
template <class R>
__device__ bool newton2(const R* a, int du, int dv, int stride, R qx, R qy, R qz, R& u, R& v, int maxit, R tol,
                        R& Dout)
{
    SD<R> o;
    eval_patch(a, du, dv, stride, u, v, o);
    GH<R> h;
    R D = grad_hess(o, qx, qy, qz, h);
    bool conv = false;
    for (int it = 0; it < maxit; ++it) {
        const bool fu = !((u <= R(0) && h.gu > R(0)) || (u >= R(1) && h.gu < R(0)));
        const bool fv = !((v <= R(0) && h.gv > R(0)) || (v >= R(1) && h.gv < R(0)));
        R su = 0, sv = 0;
        if (fu && fv) {
            R a11 = h.huu, a12 = h.huv, a22 = h.hvv;
            if (!(a11 > R(0) && a11 * a22 - a12 * a12 > R(0))) {
                a11 = h.juu;
                a12 = h.juv;
                a22 = h.jvv;
            }
            const R det = a11 * a22 - a12 * a12;
            if (a11 > R(0) && det > R(0)) {
                su = -(a22 * h.gu - a12 * h.gv) / det;
                sv = -(a11 * h.gv - a12 * h.gu) / det;
            } else {
                su = h.juu > R(0) ? -h.gu / h.juu : R(0);
                sv = h.jvv > R(0) ? -h.gv / h.jvv : R(0);
            }
        } else if (fu) {
            const R c = h.huu > R(0) ? h.huu : h.juu;
            su = c > R(0) ? -h.gu / c : R(0);
        } else if (fv) {
            const R c = h.hvv > R(0) ? h.hvv : h.jvv;
            sv = c > R(0) ? -h.gv / c : R(0);
        } else {
            conv = true;  // both coordinates held on bounds: KKT point
            break;
        }
        R lam = 1, un = u, vn = v, Dn = D;
        GH<R> hn = h;
        bool acc = false;
        for (int ls = 0; ls < 30; ++ls) {
            un = fmin(fmax(u + lam * su, R(0)), R(1));
            vn = fmin(fmax(v + lam * sv, R(0)), R(1));
            eval_patch(a, du, dv, stride, un, vn, o);
            Dn = grad_hess(o, qx, qy, qz, hn);
            if (Dn <= D) {
                acc = true;
                break;
            }
            lam *= R(0.5);
        }
        if (!acc) {
            conv = true;  // no descent left at this resolution
            break;
        }
        R step = fabs(un - u) + fabs(vn - v);
        u = un;
        v = vn;
        D = Dn;
        h = hn;
        if (step <= tol) {
            conv = true;
            break;
        }
    }
    Dout = D;
    return conv;
}

struct PoolEntry {
    int patch;
    int slot;
    float u0, v0;
};

template <class R>
struct WarpSmem {
    int cand[kCandCap];
    R cand_lb[kCandCap];
    PoolEntry pool[kPoolCap];
    double pool_D[kPoolCap];
    double pool_u[kPoolCap];
    double pool_v[kPoolCap];
    float pool_s32[kPoolCap];  // mixed: FP32 minimiser in the span pair and its squared distance
    float pool_t32[kPoolCap];
    float pool_D32[kPoolCap];
    unsigned char pool_conv32[kPoolCap];  // mixed: the FP32 stage converged
    short fin[kPoolCap];
    unsigned char pool_flags[kPoolCap];
    double q64[kQPW][3];
    float eps32[kQPW];
    float best_D32[kQPW];
    double best_D[kQPW];
    double best_u[kQPW];
    double best_v[kQPW];
    int best_patch[kQPW];
    unsigned char best_flags[kQPW];
};

// local-frame copy of a patch's power coefficients: the constant term
// becomes a(0,0) - q, formed in FP64 and rounded, so the FP32 iteration keeps
// its relative accuracy on small patches far from the origin
__device__ __forceinline__ void local_frame32(const float* a32, const double* a64_00, const double* q, int du, int dv,
                                              int stride, float* out)
{
    for (int i = 0; i <= du; ++i)
        for (int j = 0; j <= dv; ++j)
            for (int c = 0; c < 3; ++c) out[(i * stride + j) * 3 + c] = a32[(i * stride + j) * 3 + c];
    for (int c = 0; c < 3; ++c) out[c] = (float)(a64_00[c] - q[c]);
}

// Newton on the bicubic from a sampled basin; when it stops on an edge of the
// patch, a second start half a grid cell inside the patch guards against a
// minimum hidden behind a ridge of D next to that edge.  Keeps the better.
template <class R>
__device__ bool bicubic_newton(const R* c, R qx, R qy, R qz, R& u, R& v, int maxit, R tol, R hu, R hv)
{
    R D;
    bool ok = newton2<R>(c, 3, 3, 4, qx, qy, qz, u, v, maxit, tol, D);
    const bool eu = u <= R(0) || u >= R(1), ev = v <= R(0) || v >= R(1);
    if (eu || ev) {
        R u2 = eu ? (u <= R(0) ? R(0.5) * hu : R(1) - R(0.5) * hu) : u;
        R v2 = ev ? (v <= R(0) ? R(0.5) * hv : R(1) - R(0.5) * hv) : v;
        R D2;
        bool ok2 = newton2<R>(c, 3, 3, 4, qx, qy, qz, u2, v2, maxit, tol, D2);
        if (D2 < D) {
            u = u2;
            v = v2;
            ok = ok2;
        }
    }
    return ok;
}

// Newton phase over the pooled basins, then per-slot merge.
// PLAIN: FP64 Newton on the bicubic to convergence, then on the original
// span-pair patch to convergence.  MIXED: (A) FP32 Newton on the bicubic,
// then FP32 Newton on the original patch (both in the local frame); (B) best
// FP32 squared distance per query; (C) compaction of the basins within the
// FP32 margin of that best; (D) two FP64 Newton steps on the original patch,
// with the FP64 iteration as the fallback when the second step exceeds 1e-9.
template <class R, bool MIXED, int GU, int GV>
__device__ void flush_pool(const SurfQ& P, WarpSmem<R>& W, int npool, int lane)
{
    constexpr float kHu = 1.f / (GU - 1), kHv = 1.f / (GV - 1);
    if (MIXED) {
        for (int k = lane; k < npool; k += 32) {
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            float c[48];
            local_frame32(P.rec32 + (int64_t)BSPL_SREC32 * e.patch + 6,
                          P.rec64 + (int64_t)BSPL_SREC64 * e.patch + 6, q, 3, 3, 4, c);
            float uf = e.u0, vf = e.v0, Df;
            const bool ok1 = bicubic_newton<float>(c, 0.f, 0.f, 0.f, uf, vf, P.fp32_steps, 1e-7f, kHu, kHv);
            const double* pb = P.patch_box + 4 * (int64_t)e.patch;
            float s = (float)(pb[0] + uf * (pb[1] - pb[0])), t = (float)(pb[2] + vf * (pb[3] - pb[2]));
            const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
            const int pu = (int)r32[54], pv = (int)r32[55];
            const int64_t slot = P.patch_span[e.patch];
            float net[kSN * kSN * 3];
            local_frame32(P.span_net32 + (int64_t)BSPL_SPAN_NET * slot, P.span_net + (int64_t)BSPL_SPAN_NET * slot, q,
                          pu, pv, kSN, net);
            const bool ok2 = newton2<float>(net, pu, pv, kSN, 0.f, 0.f, 0.f, s, t, P.fp32_steps, 1e-7f, Df);
            W.pool_conv32[k] = ok1 && ok2;
            W.pool_s32[k] = s;
            W.pool_t32[k] = t;
            W.pool_D32[k] = Df;
            W.pool_D[k] = INFINITY;
            W.pool_flags[k] = 0;
        }
        __syncwarp();
        if (lane < kQPW) {
            float b = W.best_D32[lane];
            for (int k = 0; k < npool; ++k)
                if (W.pool[k].slot == lane) b = fminf(b, W.pool_D32[k]);
            W.best_D32[lane] = b;
        }
        __syncwarp();
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
        for (int f = lane; f < nfin; f += 32) {
            const int k = W.fin[f];
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
            const int pu = (int)r32[54], pv = (int)r32[55];
            const double* net = P.span_net + (int64_t)BSPL_SPAN_NET * P.patch_span[e.patch];
            double s = W.pool_s32[k], t = W.pool_t32[k], D;
            double s1 = s, t1 = t;
            newton2<double>(net, pu, pv, kSN, q[0], q[1], q[2], s1, t1, 1, 0.0, D);
            double s2 = s1, t2 = t1;
            newton2<double>(net, pu, pv, kSN, q[0], q[1], q[2], s2, t2, 1, 0.0, D);
            unsigned char fl = 0;
            bool ok = fabs(s2 - s1) + fabs(t2 - t1) <= 1e-9;
            s = s2;
            t = t2;
            if (!ok) {
                fl |= BSPL_Q_FALLBACK;
                ok = newton2<double>(net, pu, pv, kSN, q[0], q[1], q[2], s, t, P.newton_max, 1e-15, D);
            }
            fl |= ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
            W.pool_D[k] = D;
            W.pool_u[k] = s;
            W.pool_v[k] = t;
            W.pool_flags[k] = fl;
        }
    } else {
        for (int k = lane; k < npool; k += 32) {
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            const double* a = P.rec64 + (int64_t)BSPL_SREC64 * e.patch + 6;
            double D, u = e.u0, v = e.v0;
            bicubic_newton<double>(a, q[0], q[1], q[2], u, v, P.newton_max, 1e-15, kHu, kHv);
            const double* pb = P.patch_box + 4 * (int64_t)e.patch;
            double s = pb[0] + u * (pb[1] - pb[0]), t = pb[2] + v * (pb[3] - pb[2]);
            const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
            const int pu = (int)r32[54], pv = (int)r32[55];
            const double* net = P.span_net + (int64_t)BSPL_SPAN_NET * P.patch_span[e.patch];
            bool ok = newton2<double>(net, pu, pv, kSN, q[0], q[1], q[2], s, t, P.newton_max, 1e-15, D);
            W.pool_D[k] = D;
            W.pool_u[k] = s;
            W.pool_v[k] = t;
            W.pool_flags[k] = ok ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
        }
    }
    __syncwarp();
    if (lane < kQPW) {
        double bD = W.best_D[lane], bu = W.best_u[lane], bv = W.best_v[lane];
        int bp = W.best_patch[lane];
        unsigned char bf = W.best_flags[lane];
        for (int k = 0; k < npool; ++k) {
            if (W.pool[k].slot != lane) continue;
            const double D = W.pool_D[k];
            const int pch = W.pool[k].patch;
            const long long a = __double_as_longlong(D), b = __double_as_longlong(bD);
            if (a < b || (a == b && pch < bp)) {
                bD = D;
                bu = W.pool_u[k];
                bv = W.pool_v[k];
                bp = pch;
                bf = W.pool_flags[k];
            }
        }
        W.best_D[lane] = bD;
        W.best_u[lane] = bu;
        W.best_v[lane] = bv;
        W.best_patch[lane] = bp;
        W.best_flags[lane] = bf;
    }
    __syncwarp();
}

template <class R, int GU, int GV, bool MIXED>
__global__ void __launch_bounds__(kWarps * 32) k_query_surfaces(SurfQ P)
{
    __shared__ WarpSmem<R> smem[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<R>& W = smem[wid];
    const int64_t batch = (int64_t)blockIdx.x * kWarps + wid;
    const int64_t qbase = batch * kQPW;
    if (qbase >= P.n_q) return;
    const int nslots = (int)min((int64_t)kQPW, P.n_q - qbase);
    const R* rec = STab<R>::rec(P);
    const R* grp = STab<R>::grp(P);
    constexpr int RW = STab<R>::RW, GW = STab<R>::GW;
    constexpr int GS = GU * GV;       // samples per patch
    constexpr int PPW = 32 / GS;      // patches per warp step
    const R hu = R(1) / R(GU - 1), hv = R(1) / R(GV - 1);
    unsigned long long n_grp_tested = 0, n_seg_tested = 0, n_cand = 0, n_newton = 0;

    if (lane < kQPW) {
        W.best_D[lane] = INFINITY;
        W.best_u[lane] = 0.0;
        W.best_v[lane] = 0.0;
        W.best_patch[lane] = 0x7fffffff;
        W.best_flags[lane] = 0;
        W.best_D32[lane] = INFINITY;
    }
    int npool = 0;
    __syncwarp();

    for (int sl = 0; sl < nslots; ++sl) {
        const int64_t qi = P.order ? (int64_t)P.order[qbase + sl] : qbase + sl;
        const int c = P.q_surf[qi];
        const double qx64 = P.q_xyz[3 * qi], qy64 = P.q_xyz[3 * qi + 1], qz64 = P.q_xyz[3 * qi + 2];
        const bool bad = c < 0 || c >= P.n || !isfinite(qx64) || !isfinite(qy64) || !isfinite(qz64);
        const int cc_ = (c < 0 || c >= P.n) ? 0 : c;
        const R qx = (R)qx64, qy = (R)qy64, qz = (R)qz64;
        // distance slack: rounding of the search precision plus the certified
        // deviation of the bicubics from the original surface
        const R eps = (MIXED ? R(4e-6) : R(1e-13)) * (fabs(qx) + fabs(qy) + fabs(qz) + (R)P.diag[cc_]) +
                      (R)(P.tol_rel * P.diag[cc_]) * R(1.0001);
        if (lane == 0) {
            W.q64[sl][0] = qx64;
            W.q64[sl][1] = qy64;
            W.q64[sl][2] = qz64;
            W.eps32[sl] = (float)eps;
            if (bad) W.best_flags[sl] = BSPL_Q_INVALID;
        }
        if (bad) continue;
        const int64_t s0 = P.seg_off[c], s1 = P.seg_off[c + 1];
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];

        R ub = INFINITY;
        for (int64_t g = g0 + lane; g < g1; g += 32) ub = fmin(ub, pt_d2(grp + (int64_t)GW * g + 6, qx, qy, qz));
        ub = warp_min(ub);
        R ubs = slacked(ub, eps);
        n_grp_tested += (unsigned long long)(g1 - g0);

        int ncand = 0;
        auto grid_stage = [&]() {
            __syncwarp();
            const int sub = lane / GS, j = lane % GS;
            const int iu = j % GU, iv = j / GU;
            for (int base = 0; base < ncand; base += PPW) {
                const int k = base + sub;
                const bool act = sub < PPW && k < ncand && W.cand_lb[k] <= ubs;
                const int pch = act ? W.cand[k] : 0;
                R D = INFINITY, vu = 0, vv = 0;
                const R u = R(iu) * hu, v = R(iv) * hv;
                if (act) {
                    const R* a = rec + (int64_t)RW * pch + 6;
                    // the constant term in the patch's local frame: a(0,0) - q
                    // formed in FP64 (for the FP32 grid; exact for FP64)
                    const double* a00 = P.rec64 + (int64_t)BSPL_SREC64 * pch + 6;
                    const R off[3] = { (R)(a00[0] - qx64), (R)(a00[1] - qy64), (R)(a00[2] - qz64) };
                    R Dq = 0;
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        R x = 0;
#pragma unroll
                        for (int i = 3; i >= 0; --i) {
                            R p = 0;
#pragma unroll
                            for (int jj = 3; jj >= 0; --jj)
                                p = p * v + ((i | jj) ? a[(i * 4 + jj) * 3 + cc] : off[cc]);
                            x = x * u + p;
                        }
                        Dq += x * x;
#pragma unroll
                        for (int i = 1; i < 4; ++i)
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) vu += R(i) * fabs(a[(i * 4 + jj) * 3 + cc]);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int jj = 1; jj < 4; ++jj) vv += R(jj) * fabs(a[(i * 4 + jj) * 3 + cc]);
                    }
                    D = Dq;
                }
                // four grid neighbours (same patch sub-group)
                const R Dl = __shfl_sync(kFull, D, (lane - 1) & 31);
                const R Dr = __shfl_sync(kFull, D, (lane + 1) & 31);
                const R Dd = __shfl_sync(kFull, D, (lane - GU) & 31);
                const R Du = __shfl_sync(kFull, D, (lane + GU) & 31);
                const bool ismin = act && (iu == 0 || D <= Dl) && (iu == GU - 1 || D < Dr) &&
                                   (iv == 0 || D <= Dd) && (iv == GV - 1 || D < Du);
                ub = fmin(ub, warp_min(D));
                ubs = slacked(ub, eps);
                const R adm = slacked(ub, eps + vu * hu + vv * hv);
                const bool push = ismin && D <= adm;
                const unsigned m = __ballot_sync(kFull, push);
                const int cnt = __popc(m);
                if (cnt > 0 && npool + cnt > kPoolCap) {
                    flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
                    n_newton += npool;
                    npool = 0;
                }
                if (push) {
                    const int pos = npool + __popc(m & ((1u << lane) - 1));
                    PoolEntry e;
                    e.patch = pch;
                    e.slot = sl;
                    e.u0 = (float)u;
                    e.v0 = (float)v;
                    W.pool[pos] = e;
                }
                npool += cnt;
                __syncwarp();
            }
            n_cand += (unsigned long long)ncand;
            ncand = 0;
        };

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
                    ups = pt_d2(r + 6, qx, qy, qz);  // a00 = the patch corner S(0,0)
                }
                n_seg_tested += (unsigned long long)(se - ss);
                ub = fmin(ub, warp_min(ups));
                ubs = slacked(ub, eps);
                const bool keep = valid && lbs <= ubs;
                const unsigned km = __ballot_sync(kFull, keep);
                if (keep) {
                    const int pos = ncand + __popc(km & ((1u << lane) - 1));
                    W.cand[pos] = (int)s;
                    W.cand_lb[pos] = lbs;
                }
                ncand += __popc(km);
                if (ncand > kCandCap - 32) grid_stage();
            }
        }
        grid_stage();
    }
    if (npool > 0) {
        flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
        n_newton += npool;
    }
    __syncwarp();

    if (lane < nslots) {
        const int64_t qi = P.order ? (int64_t)P.order[qbase + lane] : qbase + lane;
        unsigned char fl = W.best_flags[lane];
        const int pch = W.best_patch[lane];
        if ((fl & BSPL_Q_INVALID) || pch == 0x7fffffff) {
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            P.uv[2 * qi] = nan;
            P.uv[2 * qi + 1] = nan;
            P.dist[qi] = nan;
            P.status[qi] = BSPL_Q_INVALID;
        } else {
            // span-local (s, t) -> original parameters through the patch's
            // parameter box and its place inside the span pair
            const double* pr = P.prange + 4 * (int64_t)pch;
            const double* pb = P.patch_box + 4 * (int64_t)pch;
            const double su = (pr[1] - pr[0]) / (pb[1] - pb[0]), sv = (pr[3] - pr[2]) / (pb[3] - pb[2]);
            const double A = pr[0] - pb[0] * su, B = pr[2] - pb[2] * sv;
            const double s = W.best_u[lane], t = W.best_v[lane];
            const double uo = s <= 0.0 ? A : (s >= 1.0 ? A + su : A + s * su);
            const double vo = t <= 0.0 ? B : (t >= 1.0 ? B + sv : B + t * sv);
            const double d = sqrt(W.best_D[lane]);
            const int c = P.q_surf[qi];
            if (P.invert && d > 1e-9 * P.diag[c]) fl |= BSPL_Q_OFF_CURVE;
            P.uv[2 * qi] = uo;
            P.uv[2 * qi + 1] = vo;
            P.dist[qi] = d;
            P.status[qi] = fl;
        }
    }
    if (P.counters) {
        unsigned long long fb = 0, nc = 0;
        if (lane < nslots) {
            fb = (W.best_flags[lane] & BSPL_Q_FALLBACK) ? 1 : 0;
            nc = (W.best_flags[lane] & BSPL_Q_NONCONV) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fb += __shfl_xor_sync(kFull, fb, o);
            nc += __shfl_xor_sync(kFull, nc, o);
        }
        if (lane == 0) {
            atomicAdd(P.counters + BSPL_CNT_QUERIES, (unsigned long long)nslots);
            atomicAdd(P.counters + BSPL_CNT_GRP_TESTED, n_grp_tested);
            atomicAdd(P.counters + BSPL_CNT_SEG_TESTED, n_seg_tested);
            atomicAdd(P.counters + BSPL_CNT_CANDIDATES, n_cand);
            atomicAdd(P.counters + BSPL_CNT_NEWTON, n_newton);
            atomicAdd(P.counters + BSPL_CNT_FALLBACK, fb);
            atomicAdd(P.counters + BSPL_CNT_NONCONV, nc);
        }
    }
}

template <class R, int GU, int GV, bool MIXED>
void launch_surf(const SurfQ& P, cudaStream_t s)
{
    int64_t batches = (P.n_q + kQPW - 1) / kQPW;
    int64_t blocks = (batches + kWarps - 1) / kWarps;
    k_query_surfaces<R, GU, GV, MIXED><<<(unsigned)blocks, kWarps * 32, 0, s>>>(P);
}

}  // namespace

bspl_status query_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf, const double* q_xyz,
                           const bspl_options* opt, int invert, double* uv, double* dist, uint8_t* status,
                           void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!segs || !segs->is_surface || n_q < 0) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    if (!q_surf || !q_xyz || !uv || !dist || !status || !segs->seg_off || !segs->grp_off || !segs->rec64 ||
        !segs->rec32 || !segs->grp64 || !segs->grp32 || !segs->prange || !segs->diag || !segs->patch_box ||
        !segs->patch_span || !segs->span_net || !segs->span_net32)
        return BSPL_EINVAL;
    if (n_q > 0x7fffffffLL || segs->capacity > 0x7fffffffLL) return BSPL_EINVAL;
    bspl_options o{};
    if (opt) o = *opt;
    int samples = o.samples ? o.samples : 32;
    if (samples != 16 && samples != 32) return BSPL_EINVAL;
    if (o.prec != BSPL_FP64 && o.prec != BSPL_MIXED) return BSPL_EINVAL;
    int sort = opt ? o.sort_queries : 1;
    SurfQ P{};
    P.seg_off = segs->seg_off;
    P.grp_off = segs->grp_off;
    P.rec64 = segs->rec64;
    P.rec32 = segs->rec32;
    P.grp64 = segs->grp64;
    P.grp32 = segs->grp32;
    P.prange = segs->prange;
    P.patch_box = segs->patch_box;
    P.patch_span = segs->patch_span;
    P.span_net = segs->span_net;
    P.span_net32 = segs->span_net32;
    P.diag = segs->diag;
    P.tol_rel = segs->tol_rel;
    P.n = segs->n;
    P.n_q = n_q;
    P.q_surf = q_surf;
    P.q_xyz = q_xyz;
    P.uv = uv;
    P.dist = dist;
    P.status = status;
    P.invert = invert;
    P.newton_max = o.newton_max > 0 ? o.newton_max : 30;
    P.fp32_steps = o.fp32_steps > 0 ? o.fp32_steps : 8;
    P.counters = (unsigned long long*)o.counters;
    P.order = nullptr;
    if (sort) {
        if (!ws || ws_bytes < query_ws_bytes(segs->n, n_q)) return BSPL_EINVAL;
        int32_t* ord = nullptr;
        if (sort_by_spline(q_surf, n_q, segs->n, ws, ws_bytes, &ord, s) != cudaSuccess) return BSPL_ECUDA;
        P.order = ord;
    }
    if (o.prec == BSPL_MIXED) {
        if (samples == 16) launch_surf<float, 4, 4, true>(P, s);
        else launch_surf<float, 8, 4, true>(P, s);
    } else {
        if (samples == 16) launch_surf<double, 4, 4, false>(P, s);
        else launch_surf<double, 8, 4, false>(P, s);
    }
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl
