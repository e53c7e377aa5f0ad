// Evaluation of the ORIGINAL B-spline curves and surfaces (Sec. 3, Eq.
// bsplinebasis) at given parameters: one thread per point, span by binary
// search, basis by the triangular Cox-de Boor recursion.  Used to place
// inversion queries on the spline.  Rational curves (per-control-point
// weights w_i): the same sums over the homogeneous points (w_i P_i, w_i),
// divided by the weight sum, and for the refinement the quotient rule.
#include <math.h>

#include "bspl_internal.cuh"

namespace bspl {

namespace {

__host__ __device__ int span_of(const double* U, int p, int m, double t)
{
    // first/last non-empty span of [t_p, t_{m+1}], then bisection
    int lo = p, hi = m;
    while (lo < m && !(U[lo] < U[lo + 1])) ++lo;
    while (hi > p && !(U[hi] < U[hi + 1])) --hi;
    if (t <= U[lo]) return lo;
    if (t >= U[hi + 1]) return hi;
    int a = lo, b = hi;  // invariant: U[a] <= t < U[b+1]
    while (a < b) {
        int mid = (a + b + 1) >> 1;
        if (U[mid] <= t) a = mid;
        else b = mid - 1;
    }
    return a;
}

template <int MP>
__host__ __device__ void basis(const double* U, int q, int p, double t, double* N)
{
    double left[MP + 1], right[MP + 1];
    N[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = t - U[q + 1 - j];
        right[j] = U[q + j] - t;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double den = right[r + 1] + left[j - r];
            double tmp = den != 0.0 ? N[r] / den : 0.0;
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
}

// C(t) of curve c, degree p <= MP, t clamped to the domain
template <int MP>
__device__ __noinline__ void eval_point(const bspl_curves& C, int c, int p, int m, double t, double* out)
{
    const double* U = C.knots + C.knot_off[c];
    t = fmin(fmax(t, U[p]), U[m + 1]);
    const int q = span_of(U, p, m, t);
    double N[MP + 1];
    basis<MP>(U, q, p, t, N);
    const double* P = C.cps + 3 * C.cp_off[c];
    for (int k = 0; k < 3; ++k) out[k] = 0.0;
    if (C.weights) {
        const double* w = C.weights + C.cp_off[c];
        double W = 0.0;
        for (int j = 0; j <= p; ++j) {
            const double nw = N[j] * w[q - p + j];
            W += nw;
            for (int k = 0; k < 3; ++k) out[k] += nw * P[3 * (q - p + j) + k];
        }
        for (int k = 0; k < 3; ++k) out[k] /= W;
    } else {
        for (int j = 0; j <= p; ++j)
            for (int k = 0; k < 3; ++k) out[k] += N[j] * P[3 * (q - p + j) + k];
    }
}

__global__ void k_eval_curves(bspl_curves C, int64_t n_q, const int32_t* __restrict__ qc,
                              const double* __restrict__ tq, double* __restrict__ xyz)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q) return;
    int c = qc[i];
    double out[3] = { NAN, NAN, NAN };
    if (c >= 0 && c < C.n) {
        int p = C.degree[c];
        int m = (int)(C.cp_off[c + 1] - C.cp_off[c]) - 1;
        if (p >= 1 && p <= kMaxCurveDegree && m >= p) {
            if (p <= kEvalMidDeg) eval_point<kEvalMidDeg>(C, c, p, m, tq[i], out);
            else eval_point<kMaxCurveDegree>(C, c, p, m, tq[i], out);
        }
    }
    for (int k = 0; k < 3; ++k) xyz[3 * i + k] = out[k];
}

// What the evaluation on one span q needs that does not depend on t: the
// reciprocals of the knot differences of the triangular Cox-de Boor
// recursion (row j, entry r: 1 / (U_{q+r+1} - U_{q+1-j+r}), 0 for an empty
// one), and the control points of C' and C'' on the span (the derivative of
// a B-spline as a B-spline of one degree less on the differences of its
// control points, Sec. 3 Eq. bsplinebasis):
//   Q_j = p (P_{q-p+j+1} - P_{q-p+j}) / (U_{q+j+1} - U_{q-p+j+1}),   j < p
//   R_j = (p-1) (Q_{j+1} - Q_j) / (U_{q+j+1} - U_{q-p+j+2}),       j < p - 1
// Both denominators span [U_q, U_{q+1}], a non-empty span, so neither is 0.
// Computed once per span for degrees up to 8, so the Newton iterations
// divide nothing; the rare higher degrees keep no cache (it would take
// kilobytes of stack per thread) and divide at every evaluation.  Rational
// curves (NC = 4): the same for the homogeneous points (w_i P_i, w_i).
template <int MP, int NC = 3>
struct SpanCache {
    static constexpr int K = MP <= 8 ? MP : 1;
    int q;
    const double* rcp;  // the curve's rows of the per-span factors below, or nullptr
    double inv[K * (K + 1) / 2];
    double H[K + 1][NC];  // the span's points (homogeneous for NC = 4)
    double Q[K][NC];
    double R[K][NC];
};

// The factors of span_prepare that depend on the knots alone, one row per
// span slot s = cp_off[c] + (q - p) of the curves of degree <= 7, shared by
// every query of a call: [0, 28) the reciprocals 1 / (U_{q+r+1} -
// U_{q+1-j+r}) at (j - 1) j / 2 + r, [28, 35) the factors p / (U_{q+j+1} -
// U_{q-p+j+1}) of C' (j < p), [35, 41) the factors (p - 1) / (U_{q+j} -
// U_{q-p+j+1}) of C'' (1 <= j < p) at 34 + j; padded to 42 doubles.
constexpr int kRcpW = 42;
constexpr int kRcpMaxDeg = 7;

__host__ __device__ __forceinline__ double rcp_inv(const double* U, int q, int j, int r)
{
    const double den = U[q + r + 1] - U[q + 1 - j + r];
    return den != 0.0 ? 1.0 / den : 0.0;
}
__host__ __device__ __forceinline__ double rcp_sq(const double* U, int p, int q, int j)
{
    return p / (U[q + j + 1] - U[q - p + j + 1]);
}
__host__ __device__ __forceinline__ double rcp_sr(const double* U, int p, int q, int j)
{
    return (p - 1) / (U[q + j] - U[q - p + j + 1]);
}

// one thread per span slot below cap (slots past the set, of degrees above
// 7 or of empty spans are left as they are: no query reads them)
__global__ void k_span_rcp(bspl_curves C, int64_t cap, double* __restrict__ tab)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= cap || s >= C.cp_off[C.n]) return;
    int64_t lo = 0, hi = C.n - 1;  // the curve: largest c with cp_off[c] <= s
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (C.cp_off[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    const int c = (int)lo, p = C.degree[c];
    const int m = (int)(C.cp_off[c + 1] - C.cp_off[c]) - 1;
    if (p < 1 || p > kRcpMaxDeg || m < p) return;
    const int q = p + (int)(s - C.cp_off[c]);
    const double* U = C.knots + C.knot_off[c];
    if (q > m || !(U[q] < U[q + 1])) return;
    double* f = tab + (int64_t)kRcpW * s;
    for (int j = 1; j <= p; ++j)
        for (int r = 0; r < j; ++r) f[(j - 1) * j / 2 + r] = rcp_inv(U, q, j, r);
    for (int j = 0; j < p; ++j) {
        f[28 + j] = rcp_sq(U, p, q, j);
        if (j >= 1) f[34 + j] = rcp_sr(U, p, q, j);
    }
}

// control point i of the curve: P_i, or (w_i P_i, w_i) for a rational one
template <int NC>
__host__ __device__ __forceinline__ double hpt(const double* P, const double* w, int i, int k)
{
    if constexpr (NC == 4) return k < 3 ? w[i] * P[3 * i + k] : w[i];
    else return P[3 * i + k];
}

// the span's factors from the shared rows when there are any (the same
// values: k_span_rcp computes them with the same operations), else here
template <int MP, int NC>
__host__ __device__ __forceinline__ void span_prepare(const double* U, const double* P, const double* w, int p, int q,
                                             SpanCache<MP, NC>& S)
{
    static_assert(MP <= 8, "span cache for low degrees only");
    S.q = q;
    const double* f = S.rcp ? S.rcp + (int64_t)kRcpW * (q - p) : nullptr;
#pragma unroll(MP <= 8 ? MP + 1 : 1)
    for (int j = 1; j <= MP; ++j) {
        if (j > p) break;
#pragma unroll(MP <= 8 ? MP + 1 : 1)
        for (int r = 0; r < MP; ++r) {
            if (r >= j) break;
            S.inv[(j - 1) * j / 2 + r] = f ? f[(j - 1) * j / 2 + r] : rcp_inv(U, q, j, r);
        }
    }
#pragma unroll(MP <= 8 ? MP + 1 : 1)
    for (int j = 0; j <= MP; ++j) {
        if (j > p) break;
        for (int k = 0; k < NC; ++k) S.H[j][k] = hpt<NC>(P, w, q - p + j, k);
    }
#pragma unroll(MP <= 8 ? MP + 1 : 1)
    for (int j = 0; j < MP; ++j) {
        if (j >= p) break;
        const double sq = f ? f[28 + j] : rcp_sq(U, p, q, j);
        for (int k = 0; k < NC; ++k) S.Q[j][k] = sq * (S.H[j + 1][k] - S.H[j][k]);
        if (j >= 1) {
            const double sr = f ? f[34 + j] : rcp_sr(U, p, q, j);
            for (int k = 0; k < NC; ++k) S.R[j - 1][k] = sr * (S.Q[j][k] - S.Q[j - 1][k]);
        }
    }
}

// C(t), C'(t) and C''(t) of a curve of degree p with control points P[0..m]:
// the basis values of degrees p, p - 1 and p - 2 at t by the triangular
// recursion (its two rows before the last kept), times the span's control
// points P, Q and R.  NC = 4: the same on the homogeneous points gives
// A, A', A'' and W, W', W'', and then C = A/W, C' = (A' - W'C)/W,
// C'' = (A'' - 2W'C' - W''C)/W.
// D2 = false: C and C' only (C2out untouched).  t inside the cached span
// (the usual case after the first evaluation) skips the span search.
template <int MP, int NC = 3, bool D2 = true>
__host__ __device__ __forceinline__ void curve_d2(const double* U, const double* P, const double* w, int p, int m, double t,
                                         SpanCache<MP, NC>& S, double* Cout, double* C1out, double* C2out)
{
    constexpr bool kCache = MP <= 8;
    int q;
    if constexpr (kCache) {
        if (S.q >= 0 && U[S.q] <= t && t < U[S.q + 1]) {
            q = S.q;
        } else {
            q = span_of(U, p, m, t);
            if (q != S.q) span_prepare<MP, NC>(U, P, w, p, q, S);
        }
    } else {
        q = span_of(U, p, m, t);
    }
    double N[MP + 1], N1[MP + 1], N2[MP + 1], left[MP + 1], right[MP + 1];
    N[0] = 1.0;
#pragma unroll(MP <= 8 ? MP + 1 : 1)
    for (int j = 1; j <= MP; ++j) {
        if (j > p) break;
        // N holds degree j - 1 here
        if (D2 && j - 1 == p - 2)
#pragma unroll(MP <= 8 ? MP + 1 : 1)
            for (int r = 0; r < MP; ++r)
                if (r < j) N2[r] = N[r];
        if (j - 1 == p - 1)
#pragma unroll(MP <= 8 ? MP + 1 : 1)
            for (int r = 0; r < MP; ++r)
                if (r < j) N1[r] = N[r];
        left[j] = t - U[q + 1 - j];
        right[j] = U[q + j] - t;
        double saved = 0.0;
#pragma unroll(MP <= 8 ? MP + 1 : 1)
        for (int r = 0; r < MP; ++r) {
            if (r >= j) break;
            double tmp;
            if constexpr (kCache) {
                tmp = N[r] * S.inv[(j - 1) * j / 2 + r];
            } else {
                const double den = right[r + 1] + left[j - r];
                tmp = den != 0.0 ? N[r] / den : 0.0;
            }
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
    double C[NC], C1[NC], C2[NC];
    for (int k = 0; k < NC; ++k) C[k] = C1[k] = C2[k] = 0.0;
    double Qp[NC];
    for (int k = 0; k < NC; ++k) Qp[k] = 0.0;
#pragma unroll(MP <= 8 ? MP + 1 : 1)
    for (int j = 0; j <= MP; ++j) {
        if (j > p) break;
        if constexpr (kCache) {
            for (int k = 0; k < NC; ++k) C[k] += N[j] * S.H[j][k];
        } else {
            for (int k = 0; k < NC; ++k) C[k] += N[j] * hpt<NC>(P, w, q - p + j, k);
        }
        if constexpr (kCache) {
            if (j < p)
                for (int k = 0; k < NC; ++k) C1[k] += N1[j] * S.Q[j][k];
            if (D2 && j + 1 < p)
                for (int k = 0; k < NC; ++k) C2[k] += N2[j] * S.R[j][k];
        } else if (j < p) {
            const double sq = p / (U[q + j + 1] - U[q - p + j + 1]);
            double Qj[NC];
            for (int k = 0; k < NC; ++k) {
                Qj[k] = sq * (hpt<NC>(P, w, q - p + j + 1, k) - hpt<NC>(P, w, q - p + j, k));
                C1[k] += N1[j] * Qj[k];
            }
            if (D2 && j >= 1) {
                const double sr = (p - 1) / (U[q + j] - U[q - p + j + 1]);
                for (int k = 0; k < NC; ++k) C2[k] += N2[j - 1] * sr * (Qj[k] - Qp[k]);
            }
            for (int k = 0; k < NC; ++k) Qp[k] = Qj[k];
        }
    }
    if constexpr (NC == 4) {
        const double iW = 1.0 / C[3], W1 = C1[3], W2 = C2[3];
        for (int k = 0; k < 3; ++k) {
            Cout[k] = C[k] * iW;
            C1out[k] = (C1[k] - W1 * Cout[k]) * iW;
            if constexpr (D2) C2out[k] = (C2[k] - 2.0 * W1 * C1out[k] - W2 * Cout[k]) * iW;
        }
    } else {
        for (int k = 0; k < 3; ++k) {
            Cout[k] = C[k];
            C1out[k] = C1[k];
            if constexpr (D2) C2out[k] = C2[k];
        }
    }
}

// Refinement on the ORIGINAL curve (the problem of Eq. projection posed on C
// itself rather than on its cubic approximant): Newton on E = (C - q).C'
// with E' = C'.C' + (C - q).C'' (Eqs. Et, E't) from the given parameter,
// each step clamped to the domain and halved until the squared distance does
// not grow (at most 12 halvings).  Converged: E is zero to its rounding (|E|
// at most 64 units of FP64 rounding of |C'| (|C - q| + |C| + |q|)), or a
// domain end where E points outward, or the step is below the resolution of
// t, or no halving of it decreases the distance, or the accepted step
// (the longest of the halvings that does not raise D) lowers the squared
// distance by at most 4 units of its rounding (a flat minimum, where t is
// ill-conditioned but D is settled), or a step moves t by at most 1e-15 of
// the domain, or q lies on the curve to the rounding of its coordinates.  A
// full Newton step that changes D by no more than D's rounding is taken and
// ends the iteration (D cannot resolve it; halving it would only spend
// evaluations).  A full step that raises D and leaves the span of t is
// first replaced by the knot it crossed (D has a kink at a C0 joint, and a
// minimum on or just across it is out of the span polynomial's reach).  The
// result's distance never exceeds the start's by more than that rounding.
//
// refine_one: the refinement of one query on a curve of degree p <= MP;
// returns whether it converged, with the final t and squared distance D.
//   NC    3, or 4 for a rational curve with weights w (rational Newton);
//   nev   evaluations of C, C', C'' made; nev1 those of C and C' alone (the
//         trial points, whose C'' is computed only when another step follows);
//   rcp   the curve's rows of the shared per-span factors, or nullptr.
template <int MP, int NC>
__host__ __device__ __noinline__ bool refine_one(const double* __restrict__ U, const double* __restrict__ P,
                                        const double* __restrict__ w, int p, int m, const double* q, int max_iter,
                                        double& t, double& D, int& nev, int& nev1, const double* rcp)
{
    const double a = U[p], b = U[m + 1];
    SpanCache<MP, NC> S;
    S.q = -1;
    S.rcp = rcp;
    double C[3], C1[3], C2[3];
    curve_d2<MP, NC>(U, P, w, p, m, t, S, C, C1, C2);
    nev = 1;
    nev1 = 0;
    bool have2 = true;  // C2 belongs to the current t
    D = 0.0;
    for (int k = 0; k < 3; ++k) D += (C[k] - q[k]) * (C[k] - q[k]);
    bool conv = false;
    for (int it = 0; it <= max_iter; ++it) {
        double E = 0.0, g = 0.0, sc = 0.0;
        for (int k = 0; k < 3; ++k) {
            E += (C[k] - q[k]) * C1[k];
            g += C1[k] * C1[k];
            sc += fabs(C1[k]) * (fabs(C[k] - q[k]) + fabs(C[k]) + fabs(q[k]));
        }
        if ((t <= a && E >= 0.0) || (t >= b && E <= 0.0) || fabs(E) <= 64.0 * 1.1102230246251565e-16 * sc) {
            conv = true;
            break;
        }
        // q on the curve to the rounding of its coordinates: D is rounding
        // noise, which no step can lower reliably
        {
            double mag = 0.0;
            for (int k = 0; k < 3; ++k) mag = fmax(mag, fabs(C[k]) + fabs(q[k]));
            const double r = 16.0 * 1.1102230246251565e-16 * mag;
            if (D <= r * r) {
                conv = true;
                break;
            }
        }
        if (it == max_iter) break;
        if (!have2) {  // another step: C'' at t (C and C' come out the same)
            curve_d2<MP, NC>(U, P, w, p, m, t, S, C, C1, C2);
            ++nev;
            have2 = true;
        }
        double h = 0.0;
        for (int k = 0; k < 3; ++k) h += (C[k] - q[k]) * C2[k];
        const double Ep = g + h;
        double dt = Ep > 0.0 ? -E / Ep : (g > 0.0 ? -E / g : 0.0);
        // a step below the resolution of t: converged
        if (!(fabs(dt) > 1e-15 * (b - a) + 4.0 * 1.1102230246251565e-16 * fabs(t))) {
            conv = true;
            break;
        }
        bool took = false;
        double tn = t, Dn = D, Cn[3], C1n[3];
        for (int hv = 0; hv < 12; ++hv, dt *= 0.5) {
            tn = fmin(fmax(t + dt, a), b);
            curve_d2<MP, NC, false>(U, P, w, p, m, tn, S, Cn, C1n, nullptr);
            ++nev1;
            Dn = 0.0;
            for (int k = 0; k < 3; ++k) Dn += (Cn[k] - q[k]) * (Cn[k] - q[k]);
            if (Dn <= D) {
                took = true;
                break;
            }
            // a full Newton step whose change of D is within D's rounding
            // (its own sum, 8 units, and the rounding of C's coordinates, 16
            // units of |C| + |q|, through 2 |C - q|) is taken: near a minimum
            // the step is Newton's and D cannot tell it apart; it ends the
            // iteration below
            if (hv == 0) {
                double mag = 0.0;
                for (int k = 0; k < 3; ++k) mag = fmax(mag, fabs(C[k]) + fabs(q[k]));
                const double noise =
                    8.0 * 1.1102230246251565e-16 * D + 32.0 * 1.1102230246251565e-16 * mag * sqrt(D);
                if (Dn <= D + noise) {
                    took = true;
                    break;
                }
                // the full step left the span of t: its model (the span's
                // polynomial) ends at the knot it crossed, where D may have a
                // kink (a C0 joint); that knot is tried before the halvings
                const int q0 = span_of(U, p, m, t);
                const double kn = tn > U[q0 + 1] ? U[q0 + 1] : (tn < U[q0] && U[q0] < t ? U[q0] : t);
                if (kn != t) {
                    double Ck[3], C1k[3];
                    curve_d2<MP, NC, false>(U, P, w, p, m, kn, S, Ck, C1k, nullptr);
                    ++nev1;
                    double Dk = 0.0;
                    for (int k = 0; k < 3; ++k) Dk += (Ck[k] - q[k]) * (Ck[k] - q[k]);
                    if (Dk <= D) {
                        tn = kn;
                        Dn = Dk;
                        for (int k = 0; k < 3; ++k) {
                            Cn[k] = Ck[k];
                            C1n[k] = C1k[k];
                        }
                        took = true;
                        break;
                    }
                }
            }
        }
        if (!took) {  // no step decreases the distance: t is a minimum to rounding
            conv = true;
            break;
        }
        const double mv = fabs(tn - t), drop = D - Dn;
        t = tn;
        D = Dn;
        for (int k = 0; k < 3; ++k) {
            C[k] = Cn[k];
            C1[k] = C1n[k];
        }
        have2 = false;
        if (mv <= 1e-15 * (b - a) || drop <= 4.0 * 1.1102230246251565e-16 * D) {
            conv = true;
            break;
        }
    }
    return conv;
}

// the refinement of query i (one thread each); evals: optional per-degree
// evaluation counts, gathered per block in shared memory
template <int NC>
__device__ __forceinline__ int refine_query(const bspl_curves& Cv, const double* __restrict__ diag, int invert,
                                            int64_t i, const int32_t* __restrict__ qc,
                                            const double* __restrict__ q_xyz, int max_iter, double* __restrict__ t_io,
                                            double* __restrict__ d_io, uint8_t* __restrict__ st_io, int& nev,
                                            int& nev1, const double* __restrict__ rcp, int64_t rcp_cap)
{
    nev = 0;
    nev1 = 0;
    const int c = qc[i];
    if (c < 0 || c >= Cv.n || (st_io[i] & BSPL_Q_INVALID)) return -1;
    const int p = Cv.degree[c];
    const int m = (int)(Cv.cp_off[c + 1] - Cv.cp_off[c]) - 1;
    if (p < 1 || p > kMaxCurveDegree || m < p) return -1;
    const double* U = Cv.knots + Cv.knot_off[c];
    const double* P = Cv.cps + 3 * Cv.cp_off[c];
    const double a = U[p], b = U[m + 1];
    double t = t_io[i];
    if (!isfinite(t)) return -1;
    t = fmin(fmax(t, a), b);
    const double q[3] = { q_xyz[3 * i], q_xyz[3 * i + 1], q_xyz[3 * i + 2] };
    double D;
    const double* w = NC == 4 ? Cv.weights + Cv.cp_off[c] : nullptr;
    // the curve's rows of the shared factors, when every one of them is there
    const double* rc = rcp && Cv.cp_off[c + 1] <= rcp_cap ? rcp + (int64_t)kRcpW * Cv.cp_off[c] : nullptr;
    const bool conv =
        p <= kRcpMaxDeg     ? refine_one<kRcpMaxDeg, NC>(U, P, w, p, m, q, max_iter, t, D, nev, nev1, rc)
        : p <= kEvalMidDeg ? refine_one<kEvalMidDeg, NC>(U, P, w, p, m, q, max_iter, t, D, nev, nev1, nullptr)
                             : refine_one<kMaxCurveDegree, NC>(U, P, w, p, m, q, max_iter, t, D, nev, nev1, nullptr);
    const double d = sqrt(D);
    uint8_t fl = st_io[i] & (uint8_t)~(BSPL_Q_CONVERGED | BSPL_Q_NONCONV | BSPL_Q_AT_END | BSPL_Q_OFF_CURVE);
    fl |= conv ? BSPL_Q_CONVERGED : BSPL_Q_NONCONV;
    if (t <= a || t >= b) fl |= BSPL_Q_AT_END;
    if (invert && diag && d > 1e-9 * diag[c]) fl |= BSPL_Q_OFF_CURVE;
    if (invert && !diag) fl |= st_io[i] & BSPL_Q_OFF_CURVE;
    t_io[i] = t;
    d_io[i] = d;
    st_io[i] = fl;
    return p;
}

// thread k refines query order[k] (queries grouped by curve), or query k
template <int NC>
__global__ void __launch_bounds__(128, 4) k_refine_curves(bspl_curves Cv, const double* __restrict__ diag, int invert, int64_t n_q,
                                const int32_t* __restrict__ qc, const double* __restrict__ q_xyz, int max_iter,
                                double* __restrict__ t_io, double* __restrict__ d_io, uint8_t* __restrict__ st_io,
                                unsigned long long* __restrict__ evals, const int32_t* __restrict__ order,
                                const double* __restrict__ rcp, int64_t rcp_cap)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int nev = 0, nev1 = 0, p = -1;
    if (k < n_q) {
        const int64_t i = order ? (int64_t)order[k] : k;
        p = refine_query<NC>(Cv, diag, invert, i, qc, q_xyz, max_iter, t_io, d_io, st_io, nev, nev1, rcp, rcp_cap);
    }
    if (evals == nullptr) return;  // uniform over the launch
    __shared__ unsigned int hist[BSPL_REFINE_EVALS];
    for (int k = threadIdx.x; k < BSPL_REFINE_EVALS; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    if (p >= 0 && nev > 0) atomicAdd(&hist[p], (unsigned int)nev);
    if (p >= 0 && nev1 > 0) atomicAdd(&hist[32 + p], (unsigned int)nev1);
    __syncthreads();
    for (int k = threadIdx.x; k < BSPL_REFINE_EVALS; k += blockDim.x)
        if (hist[k]) atomicAdd(&evals[k], (unsigned long long)hist[k]);
}

// clamped parameter, span and basis values of one direction of a surface
__device__ __noinline__ int direction_basis(const double* __restrict__ K, int p, int n, double t, double* N)
{
    t = fmin(fmax(t, K[p]), K[n]);
    int q = span_of(K, p, n - 1, t);
    basis<15>(K, q, p, t, N);
    return q;
}

__global__ void k_eval_surfaces(bspl_surfaces S, int64_t n_q, const int32_t* __restrict__ qs,
                                const double* __restrict__ uv, double* __restrict__ xyz)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q) return;
    int s = qs[i];
    double out[3] = { NAN, NAN, NAN };
    if (s >= 0 && s < S.n) {
        int pu = S.deg_u[s], pv = S.deg_v[s], nu = S.n_u[s], nv = S.n_v[s];
        if (pu >= 1 && pv >= 1 && pu <= 15 && pv <= 15 && nu > pu && nv > pv) {
            double Nu[16], Nv[16];
            const int qu = direction_basis(S.knots_u + S.knot_u_off[s], pu, nu, uv[2 * i], Nu);
            const int qv = direction_basis(S.knots_v + S.knot_v_off[s], pv, nv, uv[2 * i + 1], Nv);
            const double* P = S.cps + 3 * S.cp_off[s];
            for (int k = 0; k < 3; ++k) out[k] = 0.0;
            for (int a = 0; a <= pu; ++a)
                for (int b = 0; b <= pv; ++b) {
                    double w = Nu[a] * Nv[b];
                    const double* Pab = P + 3 * ((int64_t)(qu - pu + a) * nv + (qv - pv + b));
                    for (int k = 0; k < 3; ++k) out[k] += w * Pab[k];
                }
        }
    }
    for (int k = 0; k < 3; ++k) xyz[3 * i + k] = out[k];
}

}  // namespace

bspl_status eval_curves(const bspl_curves* c, int64_t n_q, const int32_t* qc, const double* t, double* xyz,
                        cudaStream_t s)
{
    if (!c || n_q < 0 || (n_q > 0 && (!qc || !t || !xyz))) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    k_eval_curves<<<ceil_div(n_q, 128), 128, 0, s>>>(*c, n_q, qc, t, xyz);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

size_t refine_ws_bytes(int64_t n_splines, int64_t n_cp_total, int64_t n_q)
{
    const size_t sb = (query_ws_bytes(n_splines, n_q) + 255) & ~(size_t)255;
    return sb + sizeof(double) * kRcpW * (size_t)n_cp_total;
}

bspl_status refine_curves(const bspl_curves* c, const double* diag, int invert, int64_t n_q, const int32_t* qc,
                          const double* q_xyz, int max_iter, double* t, double* dist, uint8_t* status,
                          uint64_t* evals, void* ws, size_t ws_bytes, cudaStream_t s)
{
    if (!c || n_q < 0 || max_iter < 0 || max_iter > 100) return BSPL_EINVAL;
    if (n_q > 0 && (!qc || !q_xyz || !t || !dist || !status)) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    int32_t* order = nullptr;
    double* rcp = nullptr;
    int64_t rcp_cap = 0;
    if (ws) {
        const size_t sb = query_ws_bytes(c->n, n_q);
        if (n_q > 0x7fffffffLL || c->n <= 0 || ws_bytes < sb) return BSPL_EINVAL;
        if (sort_by_spline(qc, n_q, c->n, nullptr, ws, sb, &order, nullptr, s) != cudaSuccess) return BSPL_ECUDA;
        // the per-span factors in the rest of the workspace: as many slots
        // as fit (curves whose slots do not all fit compute their own)
        const size_t off = (sb + 255) & ~(size_t)255;
        if (ws_bytes > off) {
            rcp_cap = (int64_t)((ws_bytes - off) / (sizeof(double) * kRcpW));
            rcp = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + off);
            if (rcp_cap > 0) k_span_rcp<<<ceil_div(rcp_cap, 128), 128, 0, s>>>(*c, rcp_cap, rcp);
            else rcp = nullptr;
        }
    }
    auto* ev = reinterpret_cast<unsigned long long*>(evals);
    if (c->weights)
        k_refine_curves<4><<<ceil_div(n_q, 128), 128, 0, s>>>(*c, diag, invert, n_q, qc, q_xyz,
                                                              max_iter ? max_iter : 16, t, dist, status, ev, order,
                                                              rcp, rcp_cap);
    else
        k_refine_curves<3><<<ceil_div(n_q, 128), 128, 0, s>>>(*c, diag, invert, n_q, qc, q_xyz,
                                                              max_iter ? max_iter : 16, t, dist, status, ev, order,
                                                              rcp, rcp_cap);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status eval_surfaces(const bspl_surfaces* c, int64_t n_q, const int32_t* qs, const double* uv, double* xyz,
                          cudaStream_t s)
{
    if (!c || n_q < 0 || (n_q > 0 && (!qs || !uv || !xyz))) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    k_eval_surfaces<<<ceil_div(n_q, 128), 128, 0, s>>>(*c, n_q, qs, uv, xyz);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl
