// Helpers shared by the curve query kernels: launch constants, the
// query parameter block, box and point distance bounds, E = (C - q).C' and
// its derivative (Sec. 4.2.3 Eqs. Dt, Et, E't), safeguarded and bracketed
// Newton iterations, the Bernstein form of E (degree-5 power-to-Bernstein
// matrix of Sec. 4.3) and certified isolation of its roots.
#pragma once
#include <math.h>

#include "bspl_internal.cuh"

namespace bspl {

// parameter block of the curve query kernels
struct CurveQ {
    const int64_t* seg_off;
    const int64_t* grp_off;
    const double* rec64;
    const float* rec32;
    const double* grp64;
    const float* grp32;
    const double* prange;
    const double* diag;
    int64_t n, n_q;
    const int64_t* n_q_dev;  // optional device-side query count (<= n_q)
    const int32_t* q_curve;
    const double* q_xyz;
    const int32_t* order;
    double* t;
    double* dist;
    uint8_t* status;
    int invert;
    int newton_max;
    int fp32_steps;
    unsigned long long* counters;
    unsigned long long* work;  // work-stealing batch counter (zeroed), or NULL: one batch per warp
};

// query_curves.cu: the mixed-precision grid kernel over P.order (the
// counting sort of query indices by curve, sort_by_spline, is declared in
// bspl_internal.cuh)
void launch_mixed_curves(const CurveQ& P, int occ, cudaStream_t s);

namespace {

constexpr int kQPW = 32;       // queries per warp batch
constexpr int kCandCap = 96;   // surviving segments buffered before the grid stage
constexpr int kPoolCap = 128;  // Newton basins buffered per warp
constexpr int kWarps = 4;      // warps per block
constexpr unsigned kFull = 0xffffffffu;


template <class R>
struct Tab;
template <>
struct Tab<double> {
    static __device__ const double* rec(const CurveQ& P) { return P.rec64; }
    static __device__ const double* grp(const CurveQ& P) { return P.grp64; }
    static constexpr int RW = BSPL_CREC64, GW = BSPL_GREC64;
};
template <>
struct Tab<float> {
    static __device__ const float* rec(const CurveQ& P) { return P.rec32; }
    static __device__ const float* grp(const CurveQ& P) { return P.grp32; }
    static constexpr int RW = BSPL_CREC32, GW = BSPL_GREC32;
};

template <class R>
__device__ __forceinline__ R warp_min(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// warp minimum of a non-negative float (a squared distance, or +inf): the
// bit patterns of such values order as unsigned integers, so one warp
// reduction instruction replaces the shuffle tree
__device__ __forceinline__ float warp_min_nonneg(float v)
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
    return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(v)));
#else
    return warp_min(v);  // targets without the reduction instruction (host test builds)
#endif
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

// squared-distance threshold with slack: (sqrt(ub) + eps)^2
template <class R>
__device__ __forceinline__ R slacked(R ub, R eps)
{
    R s = sqrt(ub) + eps;
    return s * s;
}

// E = (C - q).C' and E' = C'.C' + (C - q).C'' for the cubic a0 + a1 u + a2 u^2 + a3 u^3
// (Eqs. Et, E't up to the common factor 2); returns D = |C - q|^2
template <class R>
__host__ __device__ __forceinline__ R eval_E(const R* a, R qx, R qy, R qz, R u, R& E, R& Ep)
{
    R q3[3] = { qx, qy, qz };
    R D = 0, e = 0, ep = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        R a0 = a[c], a1 = a[3 + c], a2 = a[6 + c], a3 = a[9 + c];
        R C = a0 + u * (a1 + u * (a2 + u * a3)) - q3[c];
        R C1 = a1 + u * (R(2) * a2 + u * (R(3) * a3));
        R C2 = R(2) * a2 + u * (R(6) * a3);
        D += C * C;
        e += C * C1;
        ep += C1 * C1 + C * C2;
    }
    E = e;
    Ep = ep;
    return D;
}

// safeguarded Newton for a local minimum of D on the segment [0, 1], started
// in a sampled basin: a Newton step on E = D' when E' > 0, else a step of
// length hmax down the slope; every step is limited to hmax, projected onto
// [0, 1] and halved until D does not increase.  Stops at a bound where D
// rises into the segment (KKT), when no descent is left at this resolution,
// or when the step falls below tol.  Returns true unless maxit ran out.
template <class R>
struct Eps;
template <>
struct Eps<float> {
    static constexpr float v = 1.1920929e-07f;
};
template <>
struct Eps<double> {
    static constexpr double v = 2.220446049250313e-16;
};

template <class R>
__host__ __device__ bool newton_min(const R* a, R qx, R qy, R qz, R& u, R hmax, int maxit, R tol, unsigned& iters)
{
    // coordinate resolution of the evaluation: a Newton correction that moves
    // the point by less than this is rounding noise, and the iteration stops
    R scale = fabs(qx) + fabs(qy) + fabs(qz);
#pragma unroll
    for (int i = 0; i < 12; ++i) scale += fabs(a[i]);
    const R res = R(8) * Eps<R>::v * scale;
    R E, Ep;
    R D = eval_E(a, qx, qy, qz, u, E, Ep);
    for (int it = 0; it < maxit; ++it) {
        ++iters;
        if ((u <= R(0) && E >= R(0)) || (u >= R(1) && E <= R(0)) || E == R(0)) return true;
        if (Ep > R(0) && fabs(E) <= res * sqrt(Ep)) return true;
        R step = Ep > R(0) ? -E / Ep : (E > R(0) ? -hmax : hmax);
        step = fmin(fmax(step, -hmax), hmax);
        R un = u, Dn = D, En = E, Epn = Ep;
        bool acc = false;
        for (int ls = 0; ls < 24; ++ls) {
            un = fmin(fmax(u + step, R(0)), R(1));
            Dn = eval_E(a, qx, qy, qz, un, En, Epn);
            // accept a decrease of D, or, where D is locally convex, a
            // decrease of |E| (D itself is flat to rounding near a minimum,
            // E is still resolved there)
            if (Dn < D || (Ep > R(0) && fabs(En) < fabs(E))) {
                acc = true;
                break;
            }
            if (Dn == D) return true;  // no progress left at this precision
            step *= R(0.5);
        }
        if (!acc) return true;
        R moved = fabs(un - u);
        u = un;
        D = Dn;
        E = En;
        Ep = Epn;
        if (moved <= tol) return true;
    }
    return false;
}

// The two FP64 Newton steps of the mixed paths (Eqs. Et, E't): the residual
// C(u) - q, the tangent C'(u), E = (C - q).C' and the update of u in FP64
// (they fix where the root lies: for a far query an error of the tangent's
// direction moves the foot point by the distance times that error); only
// E' = |C'|^2 + (C - q).C'' and its reciprocal in FP32 (the step's relative
// error enters the next error linearly, times a step already near 1e-7).
// a64: FP64 power coefficients a0..a3 [12]; a32: FP32 a1..a3 [9].  Returns
// D = |C(u) - q|^2 in FP64 at the final u; last = size of the second step.
__host__ __device__ __forceinline__ double finish64(const double* a64, const float* a32, const double* q, double& u,
                                           double& last, unsigned& iters)
{
    double c0[3], b3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        c0[c] = a64[c] - q[c];
        b3[c] = 3.0 * a64[9 + c];
    }
    last = 1.0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        ++iters;
        const float uf = (float)u;
        double E = 0.0;
        float Ep = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double cx = fma(u, fma(u, fma(u, a64[9 + c], a64[6 + c]), a64[3 + c]), c0[c]);
            const double c1 = fma(u, fma(u, b3[c], 2.0 * a64[6 + c]), a64[3 + c]);
            E = fma(cx, c1, E);
            const float C1 = (float)c1;
            const float C2 = fmaf(uf, 6.f * a32[6 + c], 2.f * a32[3 + c]);
            Ep = fmaf(C1, C1, fmaf((float)cx, C2, Ep));
        }
        double un = Ep > 0.f ? u - E * (double)(1.f / Ep) : u;
        un = fmin(fmax(un, 0.0), 1.0);
        last = fabs(un - u);
        // without a Newton step (E' <= 0) the point is a minimum only at an
        // end where D rises into the segment (E > 0 at u = 0, E < 0 at
        // u = 1); anywhere else, a flat end included, it is not converged,
        // however small the (zero) step
        if (!(Ep > 0.f) && !((u <= 0.0 && E > 0.0) || (u >= 1.0 && E < 0.0))) last = 1.0;
        u = un;
    }
    double D = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double x = fma(u, fma(u, fma(u, a64[9 + c], a64[6 + c]), a64[3 + c]), c0[c]);
        D = fma(x, x, D);
    }
    return D;
}

// E(u)/2 = (C(u) - q).C'(u) for the cubic a0 + a1 u + a2 u^2 + a3 u^3 (Eq.
// Et), a degree-5 polynomial, in Bernstein form on [0,1]: power coefficients
// e_k, then b = T e with T_ij = C(i,j)/C(5,j) (the degree-5 power-to-
// Bernstein matrix of Sec. 4.3).  Returns the number of sign changes of b
// (zeros skipped), an upper bound of the number of roots of E in [0,1].
template <class R>
__host__ __device__ __forceinline__ int bernstein_E(const R* a, R qx, R qy, R qz, R* b)
{
    const R q3[3] = { qx, qy, qz };
    R e[6] = { 0, 0, 0, 0, 0, 0 };
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R c0 = a[c] - q3[c], c1 = a[3 + c], c2 = a[6 + c], c3 = a[9 + c];
        const R d1 = c1, d2 = R(2) * c2, d3 = R(3) * c3;  // C' = d1 + d2 u + d3 u^2
        e[0] += c0 * d1;
        e[1] += c0 * d2 + c1 * d1;
        e[2] += c0 * d3 + c1 * d2 + c2 * d1;
        e[3] += c1 * d3 + c2 * d2 + c3 * d1;
        e[4] += c2 * d3 + c3 * d2;
        e[5] += c3 * d3;
    }
    b[0] = e[0];
    b[1] = e[0] + R(0.2) * e[1];
    b[2] = e[0] + R(0.4) * e[1] + R(0.1) * e[2];
    b[3] = e[0] + R(0.6) * e[1] + R(0.3) * e[2] + R(0.1) * e[3];
    b[4] = e[0] + R(0.8) * e[1] + R(0.6) * e[2] + R(0.4) * e[3] + R(0.2) * e[4];
    b[5] = e[0] + e[1] + e[2] + e[3] + e[4] + e[5];
    int v = 0;
    R last = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (b[i] != R(0)) {
            if (last != R(0) && (b[i] > R(0)) != (last > R(0))) ++v;
            last = b[i];
        }
    }
    return v;
}

// sign of the first and of the last nonzero coefficient (0 if all are zero):
// the direction of a single sign change (zeros are skipped when counting)
template <class R>
__host__ __device__ __forceinline__ void end_signs6(const R* b, int& first, int& last)
{
    first = 0;
    last = 0;
#pragma unroll
    for (int i = 5; i >= 0; --i)
        if (b[i] != R(0)) first = b[i] > R(0) ? 1 : -1;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        if (b[i] != R(0)) last = b[i] > R(0) ? 1 : -1;
}

template <class R>
__host__ __device__ __forceinline__ int sign_changes6(const R* b)
{
    int v = 0;
    R last = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (b[i] != R(0)) {
            if (last != R(0) && (b[i] > R(0)) != (last > R(0))) ++v;
            last = b[i];
        }
    }
    return v;
}

// bracketed Newton on E for its root in [lo, hi] with E(lo) < 0 < E(hi)
template <class R>
__host__ __device__ R root_bracketed(const R* a, R qx, R qy, R qz, R lo, R hi, int maxit, R tol)
{
    R u = R(0.5) * (lo + hi);
    for (int it = 0; it < maxit; ++it) {
        R E, Ep;
        eval_E(a, qx, qy, qz, u, E, Ep);
        if (E > R(0)) hi = u;
        else if (E < R(0)) lo = u;
        else return u;
        R un = Ep > R(0) ? u - E / Ep : R(0.5) * (lo + hi);
        // a Newton step below the tolerance ends the iteration (near the
        // root it may round onto the bracket end it just moved)
        if (Ep > R(0) && fabs(un - u) <= tol) return fmin(fmax(un, lo), hi);
        if (!(un > lo && un < hi)) un = R(0.5) * (lo + hi);
        if (fabs(un - u) <= tol || hi - lo <= tol) return un;
        u = un;
    }
    return u;
}

// every local minimum of D = |C(u) - q|^2 on [0,1], certified by sign
// variations: an interval whose Bernstein coefficients of E change sign
// once holds exactly one root (a minimum when E goes from - to +); more
// changes -> split at the middle (de Casteljau); none -> no root.  The ends
// are minima when E(0) >= 0 or E(1) <= 0.  Returns the best minimiser.
// Optionally: `second` receives the second smallest D among the local
// minima found (interior minima, and the ends where E(0) >= 0 or E(1) <= 0;
// the global minimum is one of them), and `uncertain` is set when an
// examined interval has a Bernstein coefficient whose magnitude does not
// exceed its error bound (btol: the bounds of the top-level coefficients;
// an interval's coefficients are averages of its parent's, so their bounds
// are the same averages of the parent's bounds), i.e. its sign, and so the
// count of roots, is not certain at this precision.
// `second` (when given) holds three values: the second and third smallest
// D among the local minima and the minimiser of the second.
template <class R>
__host__ __device__ __noinline__ R isolate_min(const R* a, R qx, R qy, R qz, R tol, int maxit, R* second = nullptr,
                                      const R* btol = nullptr, bool* uncertain = nullptr)
{
    constexpr int kStack = 24;
    R b0[6];
    bernstein_E(a, qx, qy, qz, b0);
    R bestu = R(0), bestD;
    // the three smallest D among the local minima (and where the first two are)
    R m1 = R(INFINITY), m2 = R(INFINITY), m3 = R(INFINITY), u1 = R(0), u2 = R(0);
    auto local_min = [&](R D, R u) {
        if (D < m1) {
            m3 = m2;
            m2 = m1;
            u2 = u1;
            m1 = D;
            u1 = u;
        } else if (D < m2) {
            m3 = m2;
            m2 = D;
            u2 = u;
        } else if (D < m3) {
            m3 = D;
        }
    };
    {
        R E0, E1, Ep;
        bestD = eval_E(a, qx, qy, qz, R(0), E0, Ep);
        R D1 = eval_E(a, qx, qy, qz, R(1), E1, Ep);
        if (E0 >= R(0)) local_min(bestD, R(0));
        if (E1 <= R(0)) local_min(D1, R(1));
        if (D1 < bestD) {
            bestD = D1;
            bestu = R(1);
        }
    }
    R st_b[kStack][6], st_t[kStack][6];
    R st_lo[kStack], st_hi[kStack];
    int top = 0;
    const bool track = uncertain != nullptr && btol != nullptr;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        st_b[0][i] = b0[i];
        st_t[0][i] = track ? btol[i] : R(0);
    }
    st_lo[0] = R(0);
    st_hi[0] = R(1);
    top = 1;
    int budget = 64;  // intervals examined at most
    while (top > 0 && budget-- > 0) {
        --top;
        R b[6], bt[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            b[i] = st_b[top][i];
            bt[i] = track ? st_t[top][i] : R(0);
        }
        const R lo = st_lo[top], hi = st_hi[top];
        if (track) {
            // a coefficient inside its error bound matters only where its
            // sign could change the decision: at an end of the interval,
            // between two certain coefficients of the same sign, or in a
            // run of two or more (a lone one between - and + leaves one
            // sign change whatever its sign)
            int left = 0, run = 0;
            bool relevant = false;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const int sg = b[i] > bt[i] ? 1 : (b[i] < -bt[i] ? -1 : 0);
                if (sg == 0) {
                    if (i == 0 || i == 5) relevant = true;
                    ++run;
                } else {
                    if (run > 0 && (run > 1 || left == sg)) relevant = true;
                    run = 0;
                    left = sg;
                }
            }
            if (relevant) *uncertain = true;
        }
        const int v = sign_changes6(b);
        if (v == 0) continue;
        if (v == 1 || top + 2 > kStack || hi - lo <= tol * R(64)) {
            // a crossing from - to + (a minimum inside); an end coefficient
            // that rounded to exactly 0 does not hide it
            int sf, sl;
            end_signs6(b, sf, sl);
            if (sf < 0 && sl > 0) {
                R u = root_bracketed(a, qx, qy, qz, lo, hi, maxit, tol);
                R E, Ep;
                R D = eval_E(a, qx, qy, qz, u, E, Ep);
                local_min(D, u);
                if (D < bestD) {
                    bestD = D;
                    bestu = u;
                }
            } else if (v > 1) {
                // unresolved within the stack: try the middle as a seed
                R u = R(0.5) * (lo + hi);
                R E, Ep;
                R D = eval_E(a, qx, qy, qz, u, E, Ep);
                if (uncertain) *uncertain = true;
                local_min(D, u);
                if (D < bestD) {
                    bestD = D;
                    bestu = u;
                }
            }
            continue;
        }
        // split at the middle: left and right Bernstein coefficients (and,
        // when tracked, their error bounds)
        R w[6], L[6], Rr[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) w[i] = b[i];
        L[0] = w[0];
        Rr[5] = w[5];
#pragma unroll
        for (int r = 1; r < 6; ++r) {
#pragma unroll
            for (int i = 0; i < 6 - r; ++i) w[i] = R(0.5) * (w[i] + w[i + 1]);
            L[r] = w[0];
            Rr[5 - r] = w[5 - r];
        }
        const R mid = R(0.5) * (lo + hi);
#pragma unroll
        for (int i = 0; i < 6; ++i) st_b[top][i] = Rr[i];
        if (track) {
            R wt[6], Lt[6], Rt[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) wt[i] = bt[i];
            Lt[0] = wt[0];
            Rt[5] = wt[5];
#pragma unroll
            for (int r = 1; r < 6; ++r) {
#pragma unroll
                for (int i = 0; i < 6 - r; ++i) wt[i] = R(0.5) * (wt[i] + wt[i + 1]);
                Lt[r] = wt[0];
                Rt[5 - r] = wt[5 - r];
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                st_t[top][i] = Rt[i];
                st_t[top + 1][i] = Lt[i];
            }
        }
        st_lo[top] = mid;
        st_hi[top] = hi;
        ++top;
#pragma unroll
        for (int i = 0; i < 6; ++i) st_b[top][i] = L[i];
        st_lo[top] = lo;
        st_hi[top] = mid;
        ++top;
    }
    if (uncertain && top > 0) *uncertain = true;  // the interval budget ran out
    if (second) {
        second[0] = m2;
        second[1] = m3;
        second[2] = bestu == u1 ? u2 : u1;  // the runner-up's minimiser
    }
    return bestu;
}

// Kinds of a (query, segment) pair in the learned path, from the signs of
// the Bernstein coefficients of E (Sec. 4.3): kSeed one certified change from
// - to + (exactly one interior minimum), kEnd0 / kEnd1 none (the minimum at
// u = 0 / 1), kEnds one from + to - (a maximum inside, the minimum at an
// end), kIso two or more certified changes, kIsoU a coefficient within its
// rounding bound of zero where its sign could change the count.
enum : uint8_t { kSeed = 0, kEnd0 = 1, kEnd1 = 2, kEnds = 3, kIso = 4, kIsoU = 5 };

// Bernstein coefficients b of E/2 for the FP32 local-frame cubic c (C - q),
// and ba, the same sums over absolute values (the scale of each
// coefficient's FP32 rounding error)
__host__ __device__ __forceinline__ void bern_E32(const float* c, float* b, float* ba)
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
}

// classification of a pair from its FP32 local-frame cubic c (C - q)
__host__ __device__ __forceinline__ uint8_t classify(const float* c)
{
    float b[6], ba[6];
    bern_E32(c, b, ba);
    // sign changes of the certain coefficients; a coefficient inside its
    // rounding bound makes the pair uncertain only where its sign could
    // change the count: at an end, between two certain coefficients of the
    // same sign, or in a run of two or more
    int v = 0, last = 0, run = 0;
    bool relevant = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float tol = 1e-5f * ba[i];
        const int s = b[i] > tol ? 1 : (b[i] < -tol ? -1 : 0);
        if (s == 0) {
            if (i == 0 || i == 5) relevant = true;
            ++run;
            continue;
        }
        if (run > 0 && (run > 1 || last == s)) relevant = true;
        run = 0;
        if (last != 0 && s != last) ++v;
        last = s;
    }
    if (relevant) return kIsoU;
    const bool neg0 = b[0] < 0.f;
    if (v == 0) return neg0 ? kEnd1 : kEnd0;
    if (v == 1) return neg0 ? kSeed : kEnds;
    return kIso;
}

// lexicographic (D, seg, u) order; D >= 0, so its bit pattern orders like an integer
__device__ __forceinline__ bool better(double D, int s, double u, double bD, int bs, double bu)
{
    const long long a = __double_as_longlong(D), b = __double_as_longlong(bD);
    return a < b || (a == b && (s < bs || (s == bs && __double_as_longlong(u) < __double_as_longlong(bu))));
}

}  // namespace
}  // namespace bspl
