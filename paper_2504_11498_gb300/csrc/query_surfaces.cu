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

#include "../../include/bspl_mlp.h"
#include "bspl_internal.cuh"

namespace bspl {

cudaError_t mlp_seed_surface_pairs(const bspl_mlp* m, const int32_t* pq, const int32_t* pp, const int32_t* order,
                                   const double* q_xyz, const bspl_segments* segs, int64_t cap,
                                   const unsigned long long* n_dev, float* uv0, cudaStream_t s);
cudaError_t sort_by_spline(const int32_t* qc, int64_t n_q, int64_t n, const int32_t* rank, void* ws,
                           size_t ws_bytes, int32_t** order, unsigned long long** work, cudaStream_t s);

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
    const float* patch_net32;
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
    int cert_depth;  // refinement levels of the certification search; < 0: none
    unsigned long long* counters;
    unsigned long long* work;  // work-stealing batch counter (zeroed), or NULL: one batch per warp
    // learned seeds: mode 0 -- the sample grid seeds Newton; 1 -- the culled
    // (query, patch) candidates are written out instead (nothing else); 2 --
    // Newton starts from the network's (u, v) of each written pair (queries
    // without pairs fall back to the grid)
    int mode;
    int pair_index;          // mode 1: pair_q holds the query index (else the sorted position)
    int32_t* pair_q;
    int32_t* pair_p;         // patch of each pair
    const float* pair_uv;    // mode 2: (u, v) per pair
    int64_t pair_cap;
    unsigned long long* pair_n;  // [0] pairs written, [1] pairs found
    int32_t* q_first;        // per sorted position: first pair, or -1 (grid)
    int32_t* q_count;
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

// a00: the constant term (coordinate c at a00[c]); the local-frame callers
// pass a(0,0) - q formed in FP64 there, the others a itself
template <class R>
__device__ __noinline__ void eval_patch(const R* a, const R* a00, int du, int dv, int stride, R u, R v, SD<R>& o)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R s = 0, su = 0, sv = 0, suu = 0, suv = 0, svv = 0;
        for (int i = du; i >= 0; --i) {
            // row polynomial in v and its first two derivatives
            R p = 0, p1 = 0, p2 = 0;
            for (int j = dv; j >= 0; --j) {
                R coef = (i | j) ? a[(i * stride + j) * 3 + c] : a00[c];
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

// a parameter box [u0, u1] x [v0, v1]
template <class R>
struct Box2 {
    R u0, u1, v0, v1;
};

// projected Newton with active set and halving safeguard on a box (default
// [0,1]^2): the Newton step where the Hessian is positive definite, the
// Gauss-Newton step (J^T J, positive definite on a regular surface)
// elsewhere, so the step does not depend on how the parameters are scaled.
// A coordinate on a bound whose gradient points outward is held.  Returns
// true when converged (step below tol, KKT point on the bounds, or no descent
// left at this precision).
template <class R>
__device__ __noinline__ bool newton2(const R* a, const R* a00, int du, int dv, int stride, R qx, R qy, R qz, R& u, R& v,
                                     int maxit, R tol, R& Dout, Box2<R> bx = Box2<R>{ R(0), R(1), R(0), R(1) })
{
    SD<R> o;
    eval_patch(a, a00, du, dv, stride, u, v, o);
    GH<R> h;
    R D = grad_hess(o, qx, qy, qz, h);
    bool conv = false;
    for (int it = 0; it < maxit; ++it) {
        const bool fu = !((u <= bx.u0 && h.gu > R(0)) || (u >= bx.u1 && h.gu < R(0)));
        const bool fv = !((v <= bx.v0 && h.gv > R(0)) || (v >= bx.v1 && h.gv < R(0)));
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
            un = fmin(fmax(u + lam * su, bx.u0), bx.u1);
            vn = fmin(fmax(v + lam * sv, bx.v0), bx.v1);
            eval_patch(a, a00, du, dv, stride, un, vn, o);
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
    short slot;
    short direct;  // 1: a certification leaf: Newton on the original patch, inside the leaf
    float u0, v0;  // start in the patch's own parameters (a leaf: its centre)
    float hs, ht;  // a leaf: its half-sides (patch parameters)
};

// a cell of the certification search, in the patch's own parameters; cell
// sides are dyadic fractions (every split is by 8 or 4), exact in FP32
struct CertCell {
    float s0, s1, t0, t1;
    int depth;
};
constexpr int kStackCap = 64;

template <class R>
struct WarpSmem {
    union {
        struct {
            int cand[kCandCap];
            R cand_lb[kCandCap];
        };
        R net[kSN * kSN * 3];  // certification: the span-pair net being searched
    };
    PoolEntry pool[kPoolCap];
    double pool_D[kPoolCap];
    double pool_u[kPoolCap];
    double pool_v[kPoolCap];
    float pool_s32[kPoolCap];  // mixed: FP32 minimiser in the span pair and its squared distance
    float pool_t32[kPoolCap];
    float pool_D32[kPoolCap];
    unsigned char pool_conv32[kPoolCap];  // mixed: the FP32 stage converged (1), not (0), or left its leaf (3)
    short fin[kPoolCap];
    unsigned char pool_flags[kPoolCap];
    CertCell stk[kStackCap];
    double q64[kQPW][3];
    float eps32[kQPW];
    float eps32r[kQPW];  // rounding part of eps32 (distances on the original surface)
    int surf[kQPW];
    float best_D32[kQPW];
    double best_D[kQPW];
    double best_u[kQPW];
    double best_v[kQPW];
    int best_patch[kQPW];
    unsigned char best_flags[kQPW];
};

// Newton on the bicubic from a sampled basin; when it stops on an edge of the
// patch, a second start half a grid cell inside the patch guards against a
// minimum hidden behind a ridge of D next to that edge.  Keeps the better.
template <class R>
__device__ __noinline__ bool bicubic_newton(const R* c, const R* c00, R qx, R qy, R qz, R& u, R& v, int maxit, R tol,
                                            R hu, R hv)
{
    R D;
    bool ok = newton2<R>(c, c00, 3, 3, 4, qx, qy, qz, u, v, maxit, tol, D);
    const bool eu = u <= R(0) || u >= R(1), ev = v <= R(0) || v >= R(1);
    if (eu || ev) {
        R u2 = eu ? (u <= R(0) ? R(0.5) * hu : R(1) - R(0.5) * hu) : u;
        R v2 = ev ? (v <= R(0) ? R(0.5) * hv : R(1) - R(0.5) * hv) : v;
        R D2;
        bool ok2 = newton2<R>(c, c00, 3, 3, 4, qx, qy, qz, u2, v2, maxit, tol, D2);
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
__device__ __noinline__ void flush_pool(const SurfQ& P, WarpSmem<R>& W, int npool, int lane)
{
    constexpr float kHu = 1.f / (GU - 1), kHv = 1.f / (GV - 1);
    if (MIXED) {
        for (int k = lane; k < npool; k += 32) {
            const PoolEntry e = W.pool[k];
            const double* q = W.q64[e.slot];
            // FP32 iterations in the local frame of q: the constant term
            // a(0,0) - q is formed in FP64 and rounded, so the iteration keeps
            // its relative accuracy on small patches far from the origin
            float uf = e.u0, vf = e.v0, Df;
            bool ok1 = true, off_leaf = false;
            if (e.direct) {
                // a certification leaf: FP32 Newton on the original piece in
                // the patch's own power basis (coefficients of the patch's
                // size), inside the patch, then on to the span-pair net
                const double* a00 = P.rec64 + (int64_t)BSPL_SREC64 * e.patch + 6;
                const float off[3] = { (float)(a00[0] - q[0]), (float)(a00[1] - q[1]), (float)(a00[2] - q[2]) };
                const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
                const Box2<float> lb{ fmaxf(e.u0 - e.hs, 0.f), fminf(e.u0 + e.hs, 1.f), fmaxf(e.v0 - e.ht, 0.f),
                                      fminf(e.v0 + e.ht, 1.f) };
                const float* pn = P.patch_net32 + (int64_t)BSPL_SPAN_NET * e.patch;
                const int du = (int)r32[54], dv = (int)r32[55];
                ok1 = newton2<float>(pn, off, du, dv, kSN, 0.f, 0.f, 0.f, uf, vf, 2 * P.fp32_steps, 1e-7f, Df, lb);
                // the leaf's minimum sits on a leaf side where D still falls
                // outward (a side inside the patch, or a patch edge the surface
                // is C1 across): not a minimum of D -- the neighbouring leaf,
                // or patch, holds the one it leads to; no FP64 finish.  A
                // minimum on the side itself has a vanishing gradient and stays.
                SD<float> o;
                eval_patch<float>(pn, off, du, dv, kSN, uf, vf, o);
                GH<float> h;
                grad_hess<float>(o, 0.f, 0.f, 0.f, h);
                const int ef = (int)r32[61];
                const float thr_u = 1e-4f * sqrtf(h.juu * Df), thr_v = 1e-4f * sqrtf(h.jvv * Df);
                const bool out_u = (uf <= lb.u0 && (lb.u0 > 0.f || (ef & 1)) && h.gu > thr_u) ||
                                   (uf >= lb.u1 && (lb.u1 < 1.f || (ef & 2)) && h.gu < -thr_u);
                const bool out_v = (vf <= lb.v0 && (lb.v0 > 0.f || (ef & 4)) && h.gv > thr_v) ||
                                   (vf >= lb.v1 && (lb.v1 < 1.f || (ef & 8)) && h.gv < -thr_v);
                off_leaf = out_u || out_v;
            } else {
                const double* a00 = P.rec64 + (int64_t)BSPL_SREC64 * e.patch + 6;
                const float off[3] = { (float)(a00[0] - q[0]), (float)(a00[1] - q[1]), (float)(a00[2] - q[2]) };
                ok1 = bicubic_newton<float>(P.rec32 + (int64_t)BSPL_SREC32 * e.patch + 6, off, 0.f, 0.f, 0.f, uf, vf,
                                            P.fp32_steps, 1e-7f, kHu, kHv);
            }
            const double* pb = P.patch_box + 4 * (int64_t)e.patch;
            float s = (float)(pb[0] + uf * (pb[1] - pb[0])), t = (float)(pb[2] + vf * (pb[3] - pb[2]));
            const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
            const int pu = (int)r32[54], pv = (int)r32[55];
            const int64_t slot = P.patch_span[e.patch];
            bool ok2 = true;
            if (!e.direct) {
                const double* n00 = P.span_net + (int64_t)BSPL_SPAN_NET * slot;
                const float noff[3] = { (float)(n00[0] - q[0]), (float)(n00[1] - q[1]), (float)(n00[2] - q[2]) };
                ok2 = newton2<float>(P.span_net32 + (int64_t)BSPL_SPAN_NET * slot, noff, pu, pv, kSN, 0.f, 0.f, 0.f,
                                     s, t, P.fp32_steps, 1e-7f, Df);
            }
            W.pool_conv32[k] = off_leaf ? 3 : (ok1 && ok2);
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
                // every D32 is a distance on the ORIGINAL surface, so only
                // the FP32 rounding separates candidates
                const float sm = sqrtf(W.best_D32[sl]) + 2.f * W.eps32r[sl];
                const int cv = W.pool_conv32[k];
                take = cv != 3 && (!cv || W.pool_D32[k] <= sm * sm);
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
            newton2<double>(net, net, pu, pv, kSN, q[0], q[1], q[2], s1, t1, 1, 0.0, D);
            double s2 = s1, t2 = t1;
            newton2<double>(net, net, pu, pv, kSN, q[0], q[1], q[2], s2, t2, 1, 0.0, D);
            unsigned char fl = 0;
            bool ok = fabs(s2 - s1) + fabs(t2 - t1) <= 1e-9;
            s = s2;
            t = t2;
            if (!ok) {
                fl |= BSPL_Q_FALLBACK;
                ok = newton2<double>(net, net, pu, pv, kSN, q[0], q[1], q[2], s, t, P.newton_max, 1e-15, D);
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
            if (!e.direct) bicubic_newton<double>(a, a, q[0], q[1], q[2], u, v, P.newton_max, 1e-15, kHu, kHv);
            const double* pb = P.patch_box + 4 * (int64_t)e.patch;
            double s = pb[0] + u * (pb[1] - pb[0]), t = pb[2] + v * (pb[3] - pb[2]);
            const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * e.patch;
            const int pu = (int)r32[54], pv = (int)r32[55];
            const double* net = P.span_net + (int64_t)BSPL_SPAN_NET * P.patch_span[e.patch];
            Box2<double> bx{ 0.0, 1.0, 0.0, 1.0 };
            if (e.direct) {
                // a certification leaf: the minimum of D over the leaf
                const double w = pb[1] - pb[0], x = pb[3] - pb[2];
                bx = Box2<double>{ fmax(pb[0] + ((double)e.u0 - e.hs) * w, 0.0), fmin(pb[0] + ((double)e.u0 + e.hs) * w, 1.0),
                                   fmax(pb[2] + ((double)e.v0 - e.ht) * x, 0.0), fmin(pb[2] + ((double)e.v0 + e.ht) * x, 1.0) };
            }
            bool ok = newton2<double>(net, net, pu, pv, kSN, q[0], q[1], q[2], s, t, P.newton_max, 1e-15, D, bx);
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

// ------------------------------------------------------------------
// Certification of the minimum on the ORIGINAL surface (branch and bound).
//
// The sample grid of the bicubics finds every minimum whose basin holds a
// grid minimum; a narrower basin can be missed.  After the grid stage and
// its Newton refinement have given each query a distance D* (an upper bound
// of the minimum), every patch whose box could still hold something closer
// is searched cell by cell on the original span-pair polynomial restricted
// to the patch.  With the bounds the decomposition stored for the patch
// (the lengths of the first, second and third partials of S over the
// patch, in its own parameters), the third partials of D = |S - q|^2 are
// bounded on a cell (e.g. |D_sss| <= 2(3 |S_s||S_ss| + R |S_sss|), R the
// largest distance on the cell), and a cell of half-sides (hs, ht) around
// its centre c is discarded when
//   * a lower bound of D on the cell is at least the current upper bound:
//     the minimum over the cell of the quadratic Taylor model of D at c
//     (D, grad D and the Hessian evaluated there) less the cubic remainder,
//     or the first-order bound (|S(c) - q| - |S_s| hs - |S_t| ht)^2; or
//   * a component of grad D keeps its sign on the whole cell (|D_s(c)|
//     exceeds its largest change over the cell, from the Hessian at c and
//     the third-derivative bounds): then every point of the cell can move
//     against the gradient and lower D, so none is a minimum -- except on a
//     cell side that is a patch edge the surface is not C1 across (a C0
//     crease or the domain boundary), where the cell is kept.
// A kept cell on which the Hessian of D is positive definite throughout
// (its value at c less its largest change, from the third-derivative
// bounds) holds at most one minimum: it is discarded when it holds the
// query's best point so far (that point is then its minimum), else it is a
// leaf.  Any other kept cell is split into an 8 x 4 grid of cells along its
// longer side (one cell per lane) until cert_depth levels, after which it is
// a leaf.  Each leaf runs Newton on the original patch from its centre,
// confined to the leaf, which finds the minimum of D over the leaf (the
// Newton pool).  Every sampled distance also lowers the upper bound.  All
// quantities carry a bound on their rounding error (FP32 in the mixed path,
// FP64 in the plain one), so the discarding is safe in either precision.
template <class R>
struct URound;
template <>
struct URound<float> {
    static constexpr float v = 5.9604645e-08f;  // 2^-24
};
template <>
struct URound<double> {
    static constexpr double v = 1.1102230246251565e-16;  // 2^-53
};

template <class R>
__device__ __forceinline__ const R* span_coef(const SurfQ& P, int64_t slot);
template <>
__device__ __forceinline__ const float* span_coef<float>(const SurfQ& P, int64_t slot)
{
    return P.span_net32 + (int64_t)BSPL_SPAN_NET * slot;
}
template <>
__device__ __forceinline__ const double* span_coef<double>(const SurfQ& P, int64_t slot)
{
    return P.span_net + (int64_t)BSPL_SPAN_NET * slot;
}

// value and first partials of the span-pair polynomial minus q; the
// constant term is passed in (formed in FP64 in the local frame of q)
template <class R>
__device__ __forceinline__ void eval_d1(const R* a, const R* off, int du, int dv, R u, R v, R* S, R* Su, R* Sv)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R s = 0, su = 0, sv = 0;
        for (int i = du; i >= 0; --i) {
            R p = 0, p1 = 0;
            for (int j = dv; j >= 0; --j) {
                const R coef = (i | j) ? a[(i * kSN + j) * 3 + c] : off[c];
                p1 = p1 * v + p;
                p = p * v + coef;
            }
            su = su * u + s;
            s = s * u + p;
            sv = sv * u + p1;
        }
        S[c] = s;
        Su[c] = su;
        Sv[c] = sv;
    }
}

// minimum over the box |x| <= X, |y| <= Y of g.(x, y) + (a x^2 + 2 b x y +
// c y^2) / 2: exact where the form is positive definite (interior
// stationary point, else the best of the four sides), otherwise a lower
// bound that takes each term at its worst
template <class R>
__device__ __forceinline__ R quad_box_min(R gx, R gy, R a, R b, R c, R X, R Y)
{
    const R det = a * c - b * b;
    if (a > R(0) && det > R(0)) {
        auto q = [&](R x, R y) { return gx * x + gy * y + R(0.5) * (a * x * x + R(2) * b * x * y + c * y * y); };
        const R x0 = -(c * gx - b * gy) / det, y0 = -(a * gy - b * gx) / det;
        if (fabs(x0) <= X && fabs(y0) <= Y) return q(x0, y0);
        R m = INFINITY;
        for (int k = 0; k < 2; ++k) {
            const R sx = k ? X : -X, sy = k ? Y : -Y;
            m = fmin(m, q(sx, fmin(fmax(-(gy + b * sx) / c, -Y), Y)));
            m = fmin(m, q(fmin(fmax(-(gx + b * sy) / a, -X), X), sy));
        }
        return m;
    }
    return -fabs(gx) * X - fabs(gy) * Y +
           R(0.5) * (fmin(a, R(0)) * X * X - R(2) * fabs(b) * X * Y + fmin(c, R(0)) * Y * Y);
}

// what the cell test of one (query, patch) pair needs: the net searched and
// its constant term in the frame of q, how a cell's (s, t) maps to the net's
// parameters, the patch's derivative bounds, and the rounding bounds of the
// Horner evaluation.  FP32: the original piece in the patch's own power
// basis (coefficients of the patch's size); FP64: the span-pair net.
template <class R>
struct CellCtx {
    const R* a;
    R off[3];
    int du, dv, eflags;
    R e_org_s, e_w_s, e_org_t, e_w_t;
    R Vs, Vt, Ass, Ast, Att, Tsss, Tsst, Tstt, Tttt;
    R eS, eSs, eSt, eSss, eSst, eStt;
};

// everything but the net pointer and the rounding bounds (which need the
// weighted L1 norms of the coefficients)
template <class R, bool MIXED>
__device__ __forceinline__ void cell_ctx_init(const SurfQ& P, const double* q, int pch, CellCtx<R>& C)
{
    const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * pch;
    C.du = (int)r32[54];
    C.dv = (int)r32[55];
    C.Vs = r32[56];
    C.Vt = r32[57];
    C.Ass = r32[58];
    C.Ast = r32[59];
    C.Att = r32[60];
    C.eflags = (int)r32[61];
    C.Tsss = r32[62];
    C.Tsst = r32[63];
    C.Tstt = r32[64];
    C.Tttt = r32[65];
    const double* pb = P.patch_box + 4 * (int64_t)pch;
    C.e_org_s = MIXED ? R(0) : (R)pb[0];
    C.e_w_s = MIXED ? R(1) : (R)(pb[1] - pb[0]);
    C.e_org_t = MIXED ? R(0) : (R)pb[2];
    C.e_w_t = MIXED ? R(1) : (R)(pb[3] - pb[2]);
    const double* a64 =
        MIXED ? P.rec64 + (int64_t)BSPL_SREC64 * pch + 6 : P.span_net + (int64_t)BSPL_SPAN_NET * P.patch_span[pch];
#pragma unroll
    for (int c = 0; c < 3; ++c) C.off[c] = (R)(a64[c] - q[c]);
}

template <class R>
__device__ __forceinline__ void cell_ctx_errors(CellCtx<R>& C, const R* L /* weights 1, i, j, i(i-1), ij, j(j-1) */)
{
    const R kE = R(48) * URound<R>::v;  // Horner error factor for degree <= 7 + 7, with margin
    C.eS = kE * L[0];
    C.eSs = kE * L[1] * C.e_w_s;
    C.eSt = kE * L[2] * C.e_w_t;
    C.eSss = kE * L[3] * C.e_w_s * C.e_w_s;
    C.eSst = kE * L[4] * C.e_w_s * C.e_w_t;
    C.eStt = kE * L[5] * C.e_w_t * C.e_w_t;
}

template <class R>
__device__ __forceinline__ void l1_add(R* L, int i, int j, R x)
{
    L[0] += x;
    L[1] += R(i) * x;
    L[2] += R(j) * x;
    L[3] += R(i * (i - 1)) * x;
    L[4] += R(i * j) * x;
    L[5] += R(j * (j - 1)) * x;
}

// mixed precision (the patch's own FP32 power basis): the norms of the
// non-constant terms stored in the patch's record by the decomposition,
// plus the constant term |off| of this query (the FP64 path sums the span
// pair's net on the fly)
template <class R>
__device__ __forceinline__ void patch_l1(const SurfQ& P, int pch, const CellCtx<R>& C, R* L)
{
    const float* r32 = P.rec32 + (int64_t)BSPL_SREC32 * pch;
    L[0] = (R)r32[66] + (fabs(C.off[0]) + fabs(C.off[1]) + fabs(C.off[2]));
#pragma unroll
    for (int k = 1; k < 6; ++k) L[k] = (R)r32[66 + k];
}

struct CellRes {
    bool live, convex;
};

// The test of one cell [cs0, cs0 + hs] x [ct0, ct0 + ht] (patch parameters)
// against the upper bound ub: lower bounds of D and the gradient test
// (described above), and whether the Hessian of D is positive definite on
// the whole cell.  Dub: an upper bound of D at the cell's centre.
template <class R>
__device__ __noinline__ CellRes cell_test(const CellCtx<R>& C, float cs0, float hs, float ct0, float ht, R ub, R& Dub)
{
    constexpr R U = URound<R>::v;
    const R ds = R(0.5) * (R)hs, dt = R(0.5) * (R)ht;
    const R sc = (R)cs0 + ds, tc = (R)ct0 + dt;
    SD<R> o;
    eval_patch<R>(C.a, C.off, C.du, C.dv, kSN, C.e_org_s + sc * C.e_w_s, C.e_org_t + tc * C.e_w_t, o);
    // D, its gradient and Hessian at the centre, in the patch's parameters
    R D = 0, Ds = 0, Dt = 0, Hss = 0, Hst = 0, Htt = 0, n1 = 0, n2 = 0, m11 = 0, m12 = 0, m22 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R S = o.S[c], Ss = o.Su[c] * C.e_w_s, St = o.Sv[c] * C.e_w_t;
        const R Sss = o.Suu[c] * C.e_w_s * C.e_w_s, Sst = o.Suv[c] * C.e_w_s * C.e_w_t,
                Stt = o.Svv[c] * C.e_w_t * C.e_w_t;
        D += S * S;
        Ds += S * Ss;
        Dt += S * St;
        Hss += Ss * Ss + S * Sss;
        Hst += Ss * St + S * Sst;
        Htt += St * St + S * Stt;
        n1 += Ss * Ss;
        n2 += St * St;
        m11 += Sss * Sss;
        m12 += Sst * Sst;
        m22 += Stt * Stt;
    }
    Ds *= R(2);
    Dt *= R(2);
    Hss *= R(2);
    Hst *= R(2);
    Htt *= R(2);
    const R dist = sqrt(D), nSs = sqrt(n1), nSt = sqrt(n2);
    const R nSss = sqrt(m11), nSst = sqrt(m12), nStt = sqrt(m22);
    const R eS = C.eS, eSs = C.eSs, eSt = C.eSt, eSss = C.eSss, eSst = C.eSst, eStt = C.eStt;
    // rounding bounds of D, its gradient and Hessian from those of S - q and
    // its derivatives
    const R eD = R(2) * dist * eS + eS * eS + R(8) * U * D;
    const R eDs = R(2) * (dist * eSs + nSs * eS + eS * eSs) + R(8) * U * dist * nSs;
    const R eDt = R(2) * (dist * eSt + nSt * eS + eS * eSt) + R(8) * U * dist * nSt;
    const R eHss = R(2) * (R(2) * nSs * eSs + eSs * eSs + dist * eSss + nSss * eS + eS * eSss) +
                   R(8) * U * (n1 + dist * nSss);
    const R eHst = R(2) * (nSs * eSt + nSt * eSs + eSs * eSt + dist * eSst + nSst * eS + eS * eSst) +
                   R(8) * U * (nSs * nSt + dist * nSst);
    const R eHtt = R(2) * (R(2) * nSt * eSt + eSt * eSt + dist * eStt + nStt * eS + eS * eStt) +
                   R(8) * U * (n2 + dist * nStt);
    Dub = D + eD;
    ub = fmin(ub, Dub);
    // third partials of D on the cell
    const R reach = C.Vs * ds + C.Vt * dt;
    const R Rmax = dist + eS + reach;
    const R Ksss = R(2) * (R(3) * C.Vs * C.Ass + Rmax * C.Tsss);
    const R Ksst = R(2) * (R(2) * C.Vs * C.Ast + C.Vt * C.Ass + Rmax * C.Tsst);
    const R Kstt = R(2) * (R(2) * C.Vt * C.Ast + C.Vs * C.Att + Rmax * C.Tstt);
    const R Kttt = R(2) * (R(3) * C.Vt * C.Att + Rmax * C.Tttt);
    // lower bound of D on the cell: the quadratic model's minimum over the
    // cell, less the cubic remainder and the rounding bounds
    const R cub = (Ksss * ds * ds * ds + R(3) * Ksst * ds * ds * dt + R(3) * Kstt * ds * dt * dt +
                   Kttt * dt * dt * dt) * R(1.0 / 6.0);
    const R eq = eDs * ds + eDt * dt + R(0.5) * (eHss * ds * ds + R(2) * eHst * ds * dt + eHtt * dt * dt);
    const R qm = quad_box_min<R>(Ds, Dt, Hss, Hst, Htt, ds, dt);
    const R qscale = fabs(Ds) * ds + fabs(Dt) * dt + fabs(Hss) * ds * ds + R(2) * fabs(Hst) * ds * dt +
                     fabs(Htt) * dt * dt;
    const R lbQ = D - eD + qm - eq - cub - R(32) * U * (D + qscale);
    const R l1 = fmax(dist - eS - reach, R(0));
    const R lb = fmax(lbQ, l1 * l1 * (R(1) - R(8) * U));
    CellRes r{ lb < ub, false };
    // gradient test: a sign of D_s (D_t) fixed on the cell
    const R vs = fabs(Hss) * ds + fabs(Hst) * dt + R(0.5) * (Ksss * ds * ds + R(2) * Ksst * ds * dt + Kstt * dt * dt) +
                 eHss * ds + eHst * dt;
    const R vt = fabs(Hst) * ds + fabs(Htt) * dt + R(0.5) * (Ksst * ds * ds + R(2) * Kstt * ds * dt + Kttt * dt * dt) +
                 eHst * ds + eHtt * dt;
    if (r.live && fabs(Ds) - eDs > vs * (R(1) + R(32) * U)) {
        const bool blocked = Ds > R(0) ? (cs0 <= 0.f && !(C.eflags & 1)) : (cs0 + hs >= 1.f && !(C.eflags & 2));
        if (!blocked) r.live = false;
    }
    if (r.live && fabs(Dt) - eDt > vt * (R(1) + R(32) * U)) {
        const bool blocked = Dt > R(0) ? (ct0 <= 0.f && !(C.eflags & 4)) : (ct0 + ht >= 1.f && !(C.eflags & 8));
        if (!blocked) r.live = false;
    }
    if (r.live) {
        // Hessian positive definite on the whole cell: its centre value less
        // the largest change the third-derivative bounds allow
        const R a_lo = Hss - (Ksss * ds + Ksst * dt) - eHss, c_lo = Htt - (Kstt * ds + Kttt * dt) - eHtt;
        const R b_hi = fabs(Hst) + Ksst * ds + Kstt * dt + eHst;
        r.convex = a_lo > R(0) && c_lo > R(0) && a_lo * c_lo > b_hi * b_hi * (R(1) + R(32) * U);
    }
    return r;
}

// the query's best point, when it is a converged Newton end point (a KKT
// point of D on its span pair) on span pair `span`, lies in the cell: a
// convex cell that holds it holds nothing better
template <class R>
__device__ __forceinline__ bool holds_best(const SurfQ& P, const WarpSmem<R>& W, int sl, int64_t span,
                                           const double* pb, float cs0, float hs, float ct0, float ht)
{
    const int bp = W.best_patch[sl];
    if (bp == 0x7fffffff || !(W.best_flags[sl] & BSPL_Q_CONVERGED) || P.patch_span[bp] != span) return false;
    const double w = pb[1] - pb[0], x = pb[3] - pb[2];
    const double s0 = pb[0] + (double)cs0 * w, s1 = pb[0] + (double)(cs0 + hs) * w;
    const double t0 = pb[2] + (double)ct0 * x, t1 = pb[2] + (double)(ct0 + ht) * x;
    const double bu = W.best_u[sl], bv = W.best_v[sl];
    return bu >= s0 && bu <= s1 && bv >= t0 && bv <= t1;
}

// a leaf to the Newton pool (warp-cooperative; leaf: this lane's flag)
template <class R, bool MIXED, int GU, int GV>
__device__ __forceinline__ void push_leaves(const SurfQ& P, WarpSmem<R>& W, int sl, int pch, bool leaf, float sc,
                                            float tc, float hs2, float ht2, int lane, int& npool,
                                            unsigned long long* cnt)
{
    const unsigned lm = __ballot_sync(kFull, leaf);
    const int nl = __popc(lm);
    if (nl == 0) return;
    if (npool + nl > kPoolCap) {
        flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
        cnt[3] += (unsigned long long)npool;
        npool = 0;
    }
    if (leaf) {
        PoolEntry e;
        e.patch = pch;
        e.slot = (short)sl;
        e.direct = 1;
        e.u0 = sc;
        e.v0 = tc;
        e.hs = hs2;
        e.ht = ht2;
        W.pool[npool + __popc(lm & ((1u << lane) - 1))] = e;
    }
    npool += nl;
    if (lane == 0) cnt[1] += (unsigned long long)nl;
    __syncwarp();
}

// the cell search of one patch whose whole-patch test left it live and not
// convex: its net staged in shared memory, cells split 8 x 4 (one per lane)
template <class R, bool MIXED, int GU, int GV>
__device__ __noinline__ void certify_patch(const SurfQ& P, WarpSmem<R>& W, int sl, int pch, int lane, R& ub,
                                           int& npool, unsigned long long* cnt /* cells, leaves, overflow, newton */)
{
    const double* q = W.q64[sl];
    const int64_t span = P.patch_span[pch];
    const double* pb = P.patch_box + 4 * (int64_t)pch;
    CellCtx<R> C;
    cell_ctx_init<R, MIXED>(P, q, pch, C);
    {
        const R* ag = MIXED ? (const R*)(P.patch_net32 + (int64_t)BSPL_SPAN_NET * pch) : span_coef<R>(P, span);
        __syncwarp();
        for (int k = lane; k < kSN * kSN * 3; k += 32) W.net[k] = ag[k];
        __syncwarp();
    }
    C.a = W.net;
    R L[6] = { 0, 0, 0, 0, 0, 0 };
    if (MIXED) {
        patch_l1(P, pch, C, L);
    } else {
        const int ncoef = (C.du + 1) * (C.dv + 1) * 3;
        for (int k = lane; k < ncoef; k += 32) {
            const int i = k / ((C.dv + 1) * 3), r = k - i * (C.dv + 1) * 3, j = r / 3, c = r - 3 * j;
            l1_add(L, i, j, fabs((i | j) ? C.a[(i * kSN + j) * 3 + c] : C.off[c]));
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) L[k] += __shfl_xor_sync(kFull, L[k], o);
    }
    cell_ctx_errors(C, L);
    const int maxdepth = P.cert_depth;

    int top = 1;
    if (lane == 0) W.stk[0] = CertCell{ 0.f, 1.f, 0.f, 1.f, 0 };
    __syncwarp();
    while (top > 0) {
        const CertCell cc = W.stk[top - 1];
        __syncwarp();
        --top;
        const bool along_s = C.Vs * R(cc.s1 - cc.s0) >= C.Vt * R(cc.t1 - cc.t0);
        const int ns = along_s ? 8 : 4, nt = 32 / ns;
        const int is = lane % ns, it = lane / ns;
        const float hs = (cc.s1 - cc.s0) / (float)ns, ht = (cc.t1 - cc.t0) / (float)nt;
        const float cs0 = cc.s0 + (float)is * hs, ct0 = cc.t0 + (float)it * ht;
        R Dub;
        CellRes r = cell_test<R>(C, cs0, hs, ct0, ht, ub, Dub);
        ub = fmin(ub, warp_min(Dub));
        if (r.live && r.convex && holds_best(P, W, sl, span, pb, cs0, hs, ct0, ht)) r.live = false;
        cnt[0] += 32;
        // every lane takes the same branches here (cc.depth, top and the
        // ballot are warp-uniform), so the stack top stays uniform
        bool leaf = r.live;
        if (cc.depth < maxdepth) {
            const bool split = r.live && !r.convex;
            const unsigned m = __ballot_sync(kFull, split);
            const int k = __popc(m);
            if (top + k <= kStackCap) {
                if (split)
                    W.stk[top + __popc(m & ((1u << lane) - 1))] =
                        CertCell{ cs0, cs0 + hs, ct0, ct0 + ht, cc.depth + 1 };
                top += k;
                leaf = r.live && r.convex;
            } else if (lane == 0) {
                cnt[2] += (unsigned long long)k;  // stack full: straight to Newton (counted)
            }
        }
        push_leaves<R, MIXED, GU, GV>(P, W, sl, pch, leaf, cs0 + 0.5f * hs, ct0 + 0.5f * ht, 0.5f * hs, 0.5f * ht,
                                      lane, npool, cnt);
    }
}

// The certification search of every query slot of the warp.  Patches whose
// box lower bound does not exceed the slot's best distance are first tested
// whole, one per lane (the net read from global memory): discarded, a single
// leaf (convex), or searched cell by cell.
template <class R, bool MIXED, int GU, int GV>
__device__ __noinline__ void certify_slots(const SurfQ& P, WarpSmem<R>& W, int nslots, int lane, int& npool,
                              unsigned long long* cnt)
{
    const R* rec = STab<R>::rec(P);
    const R* grp = STab<R>::grp(P);
    constexpr int RW = STab<R>::RW, GW = STab<R>::GW;
    for (int sl = 0; sl < nslots; ++sl) {
        if ((W.best_flags[sl] & BSPL_Q_INVALID) || W.best_patch[sl] == 0x7fffffff) continue;
        const int c = W.surf[sl];
        const double* q = W.q64[sl];
        const R qx = (R)q[0], qy = (R)q[1], qz = (R)q[2];
        R ub;
        if (MIXED) ub = (R)__double2float_ru(W.best_D[sl]);
        else ub = (R)W.best_D[sl];
        const R epsb = (R)W.eps32r[sl];  // box tests in R: rounding slack
        const int64_t s0 = P.seg_off[c], s1 = P.seg_off[c + 1];
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];
        for (int64_t gb = g0; gb < g1; gb += 32) {
            const int64_t g = gb + lane;
            const R lbg = g < g1 ? box_d2(grp + (int64_t)GW * g, qx, qy, qz) : R(INFINITY);
            unsigned m = __ballot_sync(kFull, lbg <= slacked(ub, epsb));
            while (m) {
                const int jg = __ffs(m) - 1;
                m &= m - 1;
                if (!(__shfl_sync(kFull, lbg, jg) <= slacked(ub, epsb))) continue;
                const int64_t ss = s0 + (gb + jg - g0) * BSPL_GROUP;
                const int64_t se = min(ss + BSPL_GROUP, s1);
                const int64_t sg = ss + lane;
                bool cand = sg < se && box_d2(rec + (int64_t)RW * sg, qx, qy, qz) <= slacked(ub, epsb);
                // the whole-patch test, one patch per lane
                CellRes r{ false, false };
                R Dub = R(INFINITY);
                if (cand) {
                    const int pch = (int)sg;
                    CellCtx<R> C;
                    cell_ctx_init<R, MIXED>(P, q, pch, C);
                    C.a = MIXED ? (const R*)(P.patch_net32 + (int64_t)BSPL_SPAN_NET * pch)
                                : span_coef<R>(P, P.patch_span[pch]);
                    R L[6] = { 0, 0, 0, 0, 0, 0 };
                    if (MIXED) {
                        patch_l1(P, pch, C, L);
                    } else {
                        for (int i = 0; i <= C.du; ++i)
                            for (int j = 0; j <= C.dv; ++j)
                                for (int k = 0; k < 3; ++k)
                                    l1_add(L, i, j, fabs((i | j) ? C.a[(i * kSN + j) * 3 + k] : C.off[k]));
                    }
                    cell_ctx_errors(C, L);
                    r = cell_test<R>(C, 0.f, 1.f, 0.f, 1.f, ub, Dub);
                    if (r.live && r.convex &&
                        holds_best(P, W, sl, P.patch_span[pch], P.patch_box + 4 * (int64_t)pch, 0.f, 1.f, 0.f, 1.f))
                        r.live = false;
                }
                ub = fmin(ub, warp_min(Dub));
                const unsigned cm = __ballot_sync(kFull, cand);
                if (lane == 0) cnt[0] += (unsigned long long)__popc(cm);  // one cell per patch tested
                push_leaves<R, MIXED, GU, GV>(P, W, sl, (int)sg, r.live && r.convex, 0.5f, 0.5f, 0.5f, 0.5f, lane,
                                              npool, cnt);
                unsigned km = __ballot_sync(kFull, r.live && !r.convex);
                while (km) {
                    const int jp = __ffs(km) - 1;
                    km &= km - 1;
                    certify_patch<R, MIXED, GU, GV>(P, W, sl, (int)(ss + jp), lane, ub, npool, cnt);
                }
            }
        }
    }
}

template <class R, int GU, int GV, bool MIXED>
__global__ void __launch_bounds__(kWarps * 32, 4) k_query_surfaces(SurfQ P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem<R>* smem = reinterpret_cast<WarpSmem<R>*>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<R>& W = smem[wid];
    // persistent: each warp takes batches of 32 sorted queries (heaviest
    // splines first when the segments carry ranks) until none is left
    const int64_t nbatch = (P.n_q + kQPW - 1) / kQPW;
    int round = 0;
    for (int64_t batch = next_batch(P.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round); batch < nbatch;
         batch = next_batch(P.work, (int64_t)blockIdx.x * kWarps + wid, nbatch, round)) {
    const int64_t qbase = batch * kQPW;
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
            W.eps32r[sl] = (float)((MIXED ? R(4e-6) : R(1e-13)) * (fabs(qx) + fabs(qy) + fabs(qz) + (R)P.diag[cc_]));
            W.surf[sl] = cc_;
            if (bad) W.best_flags[sl] = BSPL_Q_INVALID;
        }
        if (P.mode == 1 && bad) {
            if (lane == 0 && !P.pair_index) P.q_first[qbase + sl] = -1;
            continue;
        }
        if (bad) continue;
        if (P.mode == 2 && P.q_first[qbase + sl] >= 0) {
            // the network's seeds: one Newton start per written pair
            const int f = P.q_first[qbase + sl], cnt = P.q_count[qbase + sl];
            for (int base = 0; base < cnt; base += 32) {
                const int k = base + lane;
                const bool has = k < cnt;
                const unsigned m = __ballot_sync(kFull, has);
                const int nm = __popc(m);
                if (npool + nm > kPoolCap) {
                    flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
                    n_newton += npool;
                    npool = 0;
                }
                if (has) {
                    PoolEntry e;
                    e.patch = P.pair_p[f + k];
                    e.slot = (short)sl;
                    e.direct = 0;
                    e.hs = e.ht = 0.f;
                    e.u0 = P.pair_uv ? P.pair_uv[2 * (int64_t)(f + k)] : 0.5f;
                    e.v0 = P.pair_uv ? P.pair_uv[2 * (int64_t)(f + k) + 1] : 0.5f;
                    W.pool[npool + __popc(m & ((1u << lane) - 1))] = e;
                }
                npool += nm;
                __syncwarp();
            }
            n_cand += (unsigned long long)cnt;
            continue;
        }
        const int64_t s0 = P.seg_off[c], s1 = P.seg_off[c + 1];
        const int64_t g0 = P.grp_off[c], g1 = P.grp_off[c + 1];

        R ub = INFINITY;
        for (int64_t g = g0 + lane; g < g1; g += 32) ub = fmin(ub, pt_d2(grp + (int64_t)GW * g + 6, qx, qy, qz));
        ub = warp_min(ub);
        R ubs = slacked(ub, eps);
        n_grp_tested += (unsigned long long)(g1 - g0);

        int ncand = 0;
        bool collect_over = false;
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
                    e.slot = (short)sl;
                    e.direct = 0;
                    e.hs = e.ht = 0.f;
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
                if (ncand > kCandCap - 32) {
                    if (P.mode == 1) {
                        collect_over = true;  // too many candidates: this query keeps the grid
                        break;
                    }
                    grid_stage();
                }
            }
            if (collect_over) break;
        }
        if (P.mode == 1) {
            // write this query's surviving candidates as (query, patch) pairs
            int keep_n = 0;
            unsigned long long base = 0;
            if (!collect_over) {
                for (int b0 = 0; b0 < ncand; b0 += 32)
                    keep_n += __popc(__ballot_sync(kFull, b0 + lane < ncand && W.cand_lb[b0 + lane] <= ubs));
                int ok = 0;
                if (lane == 0) {
                    atomicAdd(P.pair_n + 1, (unsigned long long)keep_n);
                    base = atomicAdd(P.pair_n, (unsigned long long)keep_n);
                    ok = base + keep_n <= (unsigned long long)P.pair_cap;
                }
                ok = __shfl_sync(kFull, ok, 0);
                base = __shfl_sync(kFull, base, 0);
                if (ok) {
                    int w = 0;
                    for (int b0 = 0; b0 < ncand; b0 += 32) {
                        const bool kp = b0 + lane < ncand && W.cand_lb[b0 + lane] <= ubs;
                        const unsigned km = __ballot_sync(kFull, kp);
                        if (kp) {
                            const int64_t j = (int64_t)base + w + __popc(km & ((1u << lane) - 1));
                            P.pair_q[j] = P.pair_index ? (int32_t)qi : (int32_t)(qbase + sl);
                            P.pair_p[j] = W.cand[b0 + lane];
                        }
                        w += __popc(km);
                    }
                } else {
                    keep_n = -1;
                }
            } else {
                keep_n = -1;
            }
            if (lane == 0 && !P.pair_index) {
                P.q_first[qbase + sl] = keep_n >= 0 ? (int32_t)base : -1;
                P.q_count[qbase + sl] = keep_n >= 0 ? keep_n : 0;
            }
            __syncwarp();
            continue;
        }
        grid_stage();
    }
    if (P.mode == 1) continue;  // collecting only
    if (npool > 0) {
        flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
        n_newton += npool;
        npool = 0;
    }
    __syncwarp();
    unsigned long long ccnt[4] = { 0, 0, 0, 0 };  // cells, leaves, overflow, newton
    if (P.cert_depth >= 0) {
        certify_slots<R, MIXED, GU, GV>(P, W, nslots, lane, npool, ccnt);
        if (npool > 0) {
            flush_pool<R, MIXED, GU, GV>(P, W, npool, lane);
            ccnt[3] += npool;
            npool = 0;
        }
        n_newton += ccnt[3];
        __syncwarp();
    }

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
            atomicAdd(P.counters + BSPL_CNT_CERT_CELLS, ccnt[0]);
            atomicAdd(P.counters + BSPL_CNT_CERT_LEAVES, ccnt[1]);
            atomicAdd(P.counters + BSPL_CNT_CERT_OVERFLOW, ccnt[2]);
        }
    }
    __syncwarp();
    }  // batches
}

template <class R, int GU, int GV, bool MIXED>
void launch_surf(const SurfQ& P, cudaStream_t s)
{
    int64_t batches = (P.n_q + kQPW - 1) / kQPW;
    int64_t blocks = (batches + kWarps - 1) / kWarps;
    const size_t smem = sizeof(WarpSmem<R>) * kWarps;
    static bool attr_set = false;  // per process; the attribute is per device function
    if (!attr_set) {
        cudaFuncSetAttribute(k_query_surfaces<R, GU, GV, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr_set = true;
    }
    if (P.work) blocks = persistent_blocks(k_query_surfaces<R, GU, GV, MIXED>, kWarps * 32, smem, blocks);
    k_query_surfaces<R, GU, GV, MIXED><<<(unsigned)blocks, kWarps * 32, smem, s>>>(P);
}

// workspace of the learned surface path: the sort's part, then the pair
// buffer (16 pairs per query on average), per-query pair ranges, counters
struct SurfPairWs {
    int32_t *pq, *pp, *first, *count;
    float* uv;
    unsigned long long* n;
    int64_t cap;
};

int64_t surf_pair_cap(int64_t n_q) { return 16 * n_q + 4096; }

bool carve_surf_pairs(void* ws, size_t bytes, int64_t n_splines, int64_t n_q, SurfPairWs& W, size_t* total)
{
    Carver cv(ws, bytes);
    cv.take<char>(query_ws_bytes(n_splines, n_q));
    W.cap = surf_pair_cap(n_q);
    W.pq = cv.take<int32_t>((size_t)W.cap);
    W.pp = cv.take<int32_t>((size_t)W.cap);
    W.uv = cv.take<float>(2 * (size_t)W.cap);
    W.first = cv.take<int32_t>((size_t)n_q);
    W.count = cv.take<int32_t>((size_t)n_q);
    W.n = cv.take<unsigned long long>(2);
    if (total) *total = cv.used + 256;
    return ws != nullptr && cv.used <= bytes && W.n != nullptr;
}

template <int GU, int GV>
bspl_status query_surfaces_learned(const SurfQ& P0, const bspl_segments* segs, const bspl_mlp* mlp, void* ws,
                                   size_t ws_bytes, cudaStream_t s)
{
    SurfPairWs PW{};
    if (!carve_surf_pairs(ws, ws_bytes, segs->n, P0.n_q, PW, nullptr)) return BSPL_EINVAL;
    SurfQ P = P0;
    int32_t* ord = nullptr;
    if (sort_by_spline(P.q_surf, P.n_q, segs->n, segs->spline_rank, ws, ws_bytes, &ord, &P.work, s) != cudaSuccess)
        return BSPL_ECUDA;
    P.order = ord;
    if (cudaMemsetAsync(PW.n, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return BSPL_ECUDA;
    P.pair_q = PW.pq;
    P.pair_p = PW.pp;
    P.pair_cap = PW.cap;
    P.pair_n = PW.n;
    P.q_first = PW.first;
    P.q_count = PW.count;
    // 1. the culled candidates of every query, as (query, patch) pairs
    SurfQ C = P;
    C.mode = 1;
    C.counters = nullptr;
    launch_surf<float, GU, GV, true>(C, s);
    // 2. the network's (u, v) start of every pair
    if (mlp && mlp_seed_surface_pairs(mlp, PW.pq, PW.pp, ord, P.q_xyz, segs, PW.cap, PW.n, PW.uv, s) != cudaSuccess)
        return BSPL_ECUDA;
    // 3. Newton from the seeds, certification, results
    SurfQ D = P;
    D.mode = 2;
    D.pair_uv = mlp ? PW.uv : nullptr;
    D.work = P.work + 1;
    launch_surf<float, GU, GV, true>(D, s);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace

size_t learned_surf_ws_bytes(int64_t n_splines, int64_t n_q)
{
    SurfPairWs W{};
    size_t total = 0;
    carve_surf_pairs(nullptr, 0, n_splines, n_q, W, &total);
    return total;
}

bspl_status query_surfaces(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf, const double* q_xyz,
                           const bspl_options* opt, int invert, double* uv, double* dist, uint8_t* status,
                           void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!segs || !segs->is_surface || n_q < 0) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    if (!q_surf || !q_xyz || !uv || !dist || !status || !segs->seg_off || !segs->grp_off || !segs->rec64 ||
        !segs->rec32 || !segs->grp64 || !segs->grp32 || !segs->prange || !segs->diag || !segs->patch_box ||
        !segs->patch_span || !segs->span_net || !segs->span_net32 || !segs->patch_net32)
        return BSPL_EINVAL;
    if (n_q > 0x7fffffffLL || segs->capacity > 0x7fffffffLL) return BSPL_EINVAL;
    bspl_options o{};
    if (opt) o = *opt;
    int samples = o.samples ? o.samples : 32;
    if (samples != 16 && samples != 32) return BSPL_EINVAL;
    if (o.prec != BSPL_FP64 && o.prec != BSPL_MIXED && o.prec != BSPL_LEARNED_MIXED) return BSPL_EINVAL;
    const bspl_mlp* mlp = (const bspl_mlp*)o.mlp;
    if (o.prec == BSPL_LEARNED_MIXED && mlp && (!mlp->params || !mlp->wbf16 || mlp->kind != BSPL_MLP_SURFACE))
        return BSPL_EINVAL;
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
    P.patch_net32 = segs->patch_net32;
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
    if (o.cert_depth > 4) return BSPL_EINVAL;
    P.cert_depth = o.cert_depth < 0 ? -1 : (o.cert_depth == 0 ? 2 : o.cert_depth);
    P.counters = (unsigned long long*)o.counters;
    P.order = nullptr;
    P.work = nullptr;
    if (o.prec == BSPL_LEARNED_MIXED) {
        if (!ws || ws_bytes < learned_surf_ws_bytes(segs->n, n_q)) return BSPL_EINVAL;
        return samples == 16 ? query_surfaces_learned<4, 4>(P, segs, mlp, ws, ws_bytes, s)
                             : query_surfaces_learned<8, 4>(P, segs, mlp, ws, ws_bytes, s);
    }
    if (sort) {
        if (!ws || ws_bytes < query_ws_bytes(segs->n, n_q)) return BSPL_EINVAL;
        int32_t* ord = nullptr;
        if (sort_by_spline(q_surf, n_q, segs->n, segs->spline_rank, ws, ws_bytes, &ord, &P.work, s) !=
            cudaSuccess)
            return BSPL_ECUDA;
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

using namespace bspl;

extern "C" bspl_status bspl_smlp_collect_pairs(const bspl_segments* segs, int64_t n_q, const int32_t* q_surf,
                                               const double* q_xyz, int64_t cap, int32_t* pair_q, int32_t* pair_patch,
                                               int64_t* n_pairs, void* ws, size_t ws_bytes, cudaStream_t stream)
{
    if (ws_misaligned(ws)) return BSPL_EINVAL;
    if (!segs || !segs->is_surface || n_q < 0 || n_q > 0x7fffffffLL || cap < 0 || !n_pairs) return BSPL_EINVAL;
    if (n_q > 0 && (!q_surf || !q_xyz || (cap > 0 && (!pair_q || !pair_patch)))) return BSPL_EINVAL;
    if (!segs->seg_off || !segs->grp_off || !segs->rec64 || !segs->rec32 || !segs->grp64 || !segs->grp32 ||
        !segs->diag || !segs->patch_box || !segs->patch_span || !segs->span_net || !segs->span_net32 ||
        !segs->patch_net32)
        return BSPL_EINVAL;
    SurfPairWs PW{};
    if (!carve_surf_pairs(ws, ws_bytes, segs->n, n_q, PW, nullptr)) return BSPL_EINVAL;
    if (cudaMemsetAsync(PW.n, 0, 2 * sizeof(unsigned long long), stream) != cudaSuccess) return BSPL_ECUDA;
    if (n_q > 0) {
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
        P.patch_net32 = segs->patch_net32;
        P.diag = segs->diag;
        P.tol_rel = segs->tol_rel;
        P.n = segs->n;
        P.n_q = n_q;
        P.q_surf = q_surf;
        P.q_xyz = q_xyz;
        P.cert_depth = -1;
        int32_t* ord = nullptr;
        if (sort_by_spline(q_surf, n_q, segs->n, segs->spline_rank, ws, ws_bytes, &ord, &P.work, stream) !=
            cudaSuccess)
            return BSPL_ECUDA;
        P.order = ord;
        P.mode = 1;
        P.pair_index = 1;
        P.pair_q = pair_q;
        P.pair_p = pair_patch;
        P.pair_cap = cap;
        P.pair_n = PW.n;
        P.q_first = PW.first;
        P.q_count = PW.count;
        launch_surf<float, 8, 4, true>(P, stream);
    }
    if (cudaMemcpyAsync(n_pairs, PW.n, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(n_pairs + 1, PW.n + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return BSPL_ECUDA;
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}
