// Error-controlled decomposition of B-spline curves and surfaces into cubic
// Bezier segments and bicubic patches (Sec. 4.2.1 and 4.2.2), in FP64;
// rational curves through their homogeneous pieces and certified Hermite
// cubics (the section "rational pieces" below).
//
// This translation unit is compiled with -fmad=false: every decision of the
// subdivision (accept a reduced piece, or split it) is made from plain IEEE
// FP64 additions, multiplications, divisions and square roots in a fixed
// order, so that the segment counts are reproducible bit for bit.
//
// Work decomposition: one thread per knot span (span pair for surfaces).  A
// span's subdivision tree is walked depth first without a stack of control
// nets: a node is identified by its depth and its path bits, and its degree-p
// piece is rebuilt from the span's Bezier piece by replaying the de Casteljau
// halvings along the path (the same halvings, in the same order, as a
// recursive walk would perform).  The walk runs twice: a counting pass, a
// prefix sum over spans, and a filling pass that writes each leaf at its
// offset.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bspl_internal.cuh"

namespace bspl {

namespace {

// ------------------------------------------------------------------ helpers

// IEEE FP64 operations with round-to-nearest and no contraction: on the
// device the _rn intrinsics, which are never merged into multiply-adds; on
// the host the plain operators (the host build has no contraction).
#ifdef __CUDA_ARCH__
__device__ __forceinline__ double fadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double fsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double fmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double fsqrt(double a) { return __dsqrt_rn(a); }
#else
inline double fadd(double a, double b) { return a + b; }
inline double fsub(double a, double b) { return a - b; }
inline double fmul(double a, double b) { return a * b; }
inline double fdiv(double a, double b) { return a / b; }
inline double fsqrt(double a) { return sqrt(a); }
#endif

__host__ __device__ double binom_d(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = fdiv(fmul(r, (double)(n - k + i)), (double)i);
    return r;
}

// g_ij = int_0^1 B_i^m B_j^n (Eq. gram)
__host__ __device__ double gram_d(int m, int n, int i, int j)
{
    double num = fmul(binom_d(m, i), binom_d(n, j));
    double den = fmul((double)(m + n + 1), binom_d(m + n, i + j));
    return fdiv(num, den);
}

// Coefficients of the cubic reduction (Eq. gram entries, p/3) and of degree
// elevation (i/(n+1), (n+1-i)/(n+1)) for degrees up to MP.  A block computes
// them once, with the same FP64 operations, instead of once per tree node.
template <int MP>
struct RedCoef {
    double g33[4][4];             // g_ij for m = n = 3
    double gp[MP + 1][2][MP + 1]; // g_{1+r, j} for m = 3, n = p
    double ap[MP + 1];            // p / 3
    double ea[MP][MP + 1];        // elevation n -> n + 1: i / (n + 1)
    double eb[MP][MP + 1];        // (n + 1 - i) / (n + 1)
    __host__ __device__ double g33_(int i, int j) const { return g33[i][j]; }
    __host__ __device__ double gp_(int p, int r, int j) const { return gp[p][r][j]; }
    __host__ __device__ double ap_(int p) const { return ap[p]; }
    __host__ __device__ double ea_(int n, int i) const { return ea[n][i]; }
    __host__ __device__ double eb_(int n, int i) const { return eb[n][i]; }
};

// The same coefficients computed where they are used (the same operations,
// so the same values): for the degrees 32..63, whose tables would not fit
// in shared memory.
constexpr int kCoefTableMaxDeg = 31;
struct CoefInline {
    __host__ __device__ double g33_(int i, int j) const { return gram_d(3, 3, i, j); }
    __host__ __device__ double gp_(int p, int r, int j) const { return j <= p ? gram_d(3, p, 1 + r, j) : 0.0; }
    __host__ __device__ double ap_(int p) const { return fdiv((double)p, 3.0); }
    __host__ __device__ double ea_(int n, int i) const { return fdiv((double)i, (double)(n + 1)); }
    __host__ __device__ double eb_(int n, int i) const { return fdiv((double)(n + 1 - i), (double)(n + 1)); }
};

// every thread of the block must call this
template <int MP>
__device__ void fill_coef(RedCoef<MP>& cf)
{
    constexpr int NG = 16, NP = (MP + 1) * 2 * (MP + 1), NA = MP + 1, NE = MP * (MP + 1);
    for (int t = threadIdx.x; t < NG + NP + NA + NE; t += blockDim.x) {
        if (t < NG) {
            cf.g33[t >> 2][t & 3] = gram_d(3, 3, t >> 2, t & 3);
        } else if (t < NG + NP) {
            const int u = t - NG, p = u / (2 * (MP + 1)), r = (u / (MP + 1)) & 1, j = u % (MP + 1);
            cf.gp[p][r][j] = j <= p ? gram_d(3, p, 1 + r, j) : 0.0;
        } else if (t < NG + NP + NA) {
            const int p = t - NG - NP;
            cf.ap[p] = fdiv((double)p, 3.0);
        } else {
            const int u = t - NG - NP - NA, n = u / (MP + 1), i = u % (MP + 1);
            cf.ea[n][i] = fdiv((double)i, (double)(n + 1));
            cf.eb[n][i] = fdiv((double)(n + 1 - i), (double)(n + 1));
        }
    }
    __syncthreads();
}

// Bezier piece of knot span q from the p+1 control points starting at
// P_{q-p} (stride 3*pstride doubles between points): local power basis of
// N_{q-p..q,p} in u = (t - t_q)/(t_{q+1} - t_q) by the Cox-de Boor recursion
// on polynomials (the product M_{q,p,T} A_{q,p,T}), coefficients c = (M A) P,
// Bezier points Q = B_p^{-1} c with (B_p^{-1})_{ij} = C(i,j)/C(p,j).
// NC = 4: the homogeneous points (w_j P_j, w_j) of a rational curve, wl the
// weights (the route is linear in the points); Q is then [p+1][4].
template <int MP, int NC = 3>
__host__ __device__ void span_bezier(int p, const double* __restrict__ U, int q, const double* __restrict__ Pl,
                                     int64_t pstride, double* Q, const double* __restrict__ wl = nullptr)
{
    double poly[MP + 1][MP + 1], nw[MP + 1][MP + 1];
    double du = fsub(U[q + 1], U[q]);
    poly[0][0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        for (int j = 0; j <= k; ++j) {
            int i = q - k + j;
            for (int e = 0; e <= k; ++e) nw[j][e] = 0.0;
            if (j >= 1) {
                double den = fsub(U[i + k], U[i]);
                if (den != 0.0) {
                    double a = fdiv(fsub(U[q], U[i]), den), b = fdiv(du, den);
                    for (int e = 0; e <= k - 1; ++e) {
                        nw[j][e] = fadd(nw[j][e], fmul(a, poly[j - 1][e]));
                        nw[j][e + 1] = fadd(nw[j][e + 1], fmul(b, poly[j - 1][e]));
                    }
                }
            }
            if (j <= k - 1) {
                double den = fsub(U[i + k + 1], U[i + 1]);
                if (den != 0.0) {
                    double a = fdiv(fsub(U[i + k + 1], U[q]), den), b = fdiv(-du, den);
                    for (int e = 0; e <= k - 1; ++e) {
                        nw[j][e] = fadd(nw[j][e], fmul(a, poly[j][e]));
                        nw[j][e + 1] = fadd(nw[j][e + 1], fmul(b, poly[j][e]));
                    }
                }
            }
        }
        for (int j = 0; j <= k; ++j)
            for (int e = 0; e <= k; ++e) poly[j][e] = nw[j][e];
    }
    double cc[MP + 1][NC];
    for (int e = 0; e <= p; ++e)
        for (int c = 0; c < NC; ++c) {
            double s = 0.0;
            for (int j = 0; j <= p; ++j) {
                double v;
                if constexpr (NC == 4) v = c < 3 ? fmul(wl[j], Pl[3 * pstride * j + c]) : wl[j];
                else v = Pl[3 * pstride * j + c];
                s = fadd(s, fmul(poly[j][e], v));
            }
            cc[e][c] = s;
        }
    for (int i = 0; i <= p; ++i)
        for (int c = 0; c < NC; ++c) {
            double s = 0.0;
            for (int e = 0; e <= i; ++e) s = fadd(s, fmul(fdiv(binom_d(i, e), binom_d(p, e)), cc[e][c]));
            Q[NC * i + c] = s;
        }
}

// Bezier points of span q from the blossom of the span's polynomial, for
// degrees above 7 (where the matrix route's power-basis coefficients, of
// the size of C(p, p/2), take that many digits: 2e-10 of the control
// points' size at degree 15, 1e-2 at 31): Q_j is the blossom
// at (t_q x (p - j), t_{q+1} x j), by de Boor's algorithm with the
// arguments in that order, d_i <- (1 - a) d_{i-1} + a d_i with a = (x -
// t_i) / (t_{i+p+1-r} - t_i) in [0, 1]; NC = 4: the homogeneous points
// (w_i P_i, w_i), wl the weights
template <int MP, int NC = 3>
__host__ __device__ void span_blossom(int p, const double* __restrict__ U, int q, const double* __restrict__ Pl,
                                      double* Q, const double* __restrict__ wl = nullptr)
{
    double d[MP + 1][NC];
    for (int j = 0; j <= p; ++j) {
        for (int i = 0; i <= p; ++i)
            for (int c = 0; c < NC; ++c) {
                if constexpr (NC == 4) d[i][c] = c < 3 ? fmul(wl[i], Pl[3 * i + c]) : wl[i];
                else d[i][c] = Pl[3 * i + c];
            }
        for (int r = 1; r <= p; ++r) {
            const double x = r <= p - j ? U[q] : U[q + 1];
            for (int i = p; i >= r; --i) {
                const int g = q - p + i;
                const double a = fdiv(fsub(x, U[g]), fsub(U[g + p + 1 - r], U[g]));
                const double b = fsub(1.0, a);
                for (int c = 0; c < NC; ++c) d[i][c] = fadd(fmul(b, d[i - 1][c]), fmul(a, d[i][c]));
            }
        }
        for (int c = 0; c < NC; ++c) Q[NC * j + c] = d[p][c];
    }
}

// degree n -> n+1 (exact degree elevation); Q and E indexed with stride s (points)
template <int MP, class CF>
__host__ __device__ void elevate(int n, const double* Q, double* E, int s, const CF& cf)
{
    for (int c = 0; c < 3; ++c) {
        E[c] = Q[c];
        E[(n + 1) * s + c] = Q[n * s + c];
    }
    for (int i = 1; i <= n; ++i) {
        const double a = cf.ea_(n, i), b = cf.eb_(n, i);
        for (int c = 0; c < 3; ++c) E[i * s + c] = fadd(fmul(a, Q[(i - 1) * s + c]), fmul(b, Q[i * s + c]));
    }
}

// G1-continuous L2-optimal reduction p > 3 -> 3 (Eqs. G1-condition, epsl,
// differentiatedelta0/1).  The 2x2 normal equations are the ones obtained
// from eps: delta0 (A0.d0) + delta1 (A1.d0) = V1.d0 and
// delta0 (B0.d1) + delta1 (B1.d1) = V2.d1, A0 = a g11 d0, A1 = -a g12 d1,
// B0 = a g21 d0, B1 = -a g22 d1, a = p/3; degenerate systems fall back to
// delta0 = delta1 = 1.
template <int MP, class CF>
__host__ __device__ void reduce_g1(int p, const double* Q, int s, double* R, int rs, const CF& cf)
{
    const double* Q0 = Q;
    const double* Q1 = Q + s;
    const double* Qm = Q + (p - 1) * s;
    const double* Qp = Q + p * s;
    const double a = cf.ap_(p);
    const double g11 = cf.g33_(1, 1), g12 = cf.g33_(1, 2);
    const double g21 = cf.g33_(2, 1), g22 = cf.g33_(2, 2);
    const double g10 = cf.g33_(1, 0), g13 = cf.g33_(1, 3);
    const double g20 = cf.g33_(2, 0), g23 = cf.g33_(2, 3);
    double d0[3], d1[3], V1[3], V2[3];
    for (int c = 0; c < 3; ++c) {
        d0[c] = fsub(Q1[c], Q0[c]);
        d1[c] = fsub(Qp[c], Qm[c]);
        double s1 = 0.0, s2 = 0.0;
        for (int j = 0; j <= p; ++j) {
            s1 = fadd(s1, fmul(cf.gp_(p, 0, j), Q[j * s + c]));
            s2 = fadd(s2, fmul(cf.gp_(p, 1, j), Q[j * s + c]));
        }
        double t1 = fadd(fadd(fadd(fmul(g10, Q0[c]), fmul(g11, Q0[c])), fmul(g12, Qp[c])), fmul(g13, Qp[c]));
        double t2 = fadd(fadd(fadd(fmul(g20, Q0[c]), fmul(g21, Q0[c])), fmul(g22, Qp[c])), fmul(g23, Qp[c]));
        V1[c] = fsub(s1, t1);
        V2[c] = fsub(s2, t2);
    }
    double A0[3], A1[3], B0[3], B1[3];
    for (int c = 0; c < 3; ++c) {
        A0[c] = fmul(fmul(a, g11), d0[c]);
        A1[c] = fmul(fmul(-a, g12), d1[c]);
        B0[c] = fmul(fmul(a, g21), d0[c]);
        B1[c] = fmul(fmul(-a, g22), d1[c]);
    }
    double a11 = fadd(fadd(fmul(A0[0], d0[0]), fmul(A0[1], d0[1])), fmul(A0[2], d0[2]));
    double a12 = fadd(fadd(fmul(A1[0], d0[0]), fmul(A1[1], d0[1])), fmul(A1[2], d0[2]));
    double b1 = fadd(fadd(fmul(V1[0], d0[0]), fmul(V1[1], d0[1])), fmul(V1[2], d0[2]));
    double a21 = fadd(fadd(fmul(B0[0], d1[0]), fmul(B0[1], d1[1])), fmul(B0[2], d1[2]));
    double a22 = fadd(fadd(fmul(B1[0], d1[0]), fmul(B1[1], d1[1])), fmul(B1[2], d1[2]));
    double b2 = fadd(fadd(fmul(V2[0], d1[0]), fmul(V2[1], d1[1])), fmul(V2[2], d1[2]));
    double det = fsub(fmul(a11, a22), fmul(a12, a21));
    double dl0 = fdiv(fsub(fmul(b1, a22), fmul(a12, b2)), det);
    double dl1 = fdiv(fsub(fmul(a11, b2), fmul(b1, a21)), det);
    bool ok = (det != 0.0) && (fabs(det) > fmul(1e-12, fabs(fmul(a11, a22)))) && isfinite(dl0) && isfinite(dl1) &&
              dl0 > 0.0 && dl1 > 0.0;
    if (!ok) {
        dl0 = 1.0;
        dl1 = 1.0;
    }
    double s0 = fmul(a, dl0), s1 = fmul(a, dl1);
    for (int c = 0; c < 3; ++c) {
        R[c] = Q0[c];
        R[rs + c] = fadd(Q0[c], fmul(s0, d0[c]));
        R[2 * rs + c] = fsub(Qp[c], fmul(s1, d1[c]));
        R[3 * rs + c] = Qp[c];
    }
}

template <int MP, class CF>
__host__ __device__ void to_cubic(int p, const double* Q, int s, double* R, int rs, const CF& cf)
{
    if (p == 3) {
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) R[i * rs + c] = Q[i * s + c];
    } else if (p > 3) {
        reduce_g1<MP>(p, Q, s, R, rs, cf);
    } else {
        double w[12], x[12];
        for (int i = 0; i <= p; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Q[i * s + c];
        for (int n = p; n < 3; ++n) {
            elevate<MP>(n, w, x, 3, cf);
            for (int i = 0; i <= n + 1; ++i)
                for (int c = 0; c < 3; ++c) w[3 * i + c] = x[3 * i + c];
        }
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) R[i * rs + c] = w[3 * i + c];
    }
}

// max_i |Q_i - (R elevated to p)_i|^2 (certified deviation bound)
template <int MP, class CF>
__host__ __device__ double bound2_curve(int p, const double* Q, int s, const double* R, int rs, const CF& cf)
{
    double w[(MP + 1) * 3], x[(MP + 1) * 3];
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c) w[3 * i + c] = R[i * rs + c];
    for (int n = 3; n < p; ++n) {
        elevate<MP>(n, w, x, 3, cf);
        for (int i = 0; i <= n + 1; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = x[3 * i + c];
    }
    double b = 0.0;
    for (int i = 0; i <= p; ++i) {
        double dx = fsub(Q[i * s + 0], w[3 * i]), dy = fsub(Q[i * s + 1], w[3 * i + 1]),
               dz = fsub(Q[i * s + 2], w[3 * i + 2]);
        double e = fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
        if (e > b) b = e;
    }
    return b;
}

// de Casteljau halving at 1/2; keeps the left (side = 0) or right (side = 1)
// half in place.  Identical arithmetic to computing both halves at once.
// (NC = 4: homogeneous points, whose halving is the same linear map)
template <int MP, int NC = 3>
__host__ __device__ void halve_keep(int p, double* Q, int s, int side)
{
    double w[(MP + 1) * NC], keep[(MP + 1) * NC];
    for (int i = 0; i <= p; ++i)
        for (int c = 0; c < NC; ++c) w[NC * i + c] = Q[i * s + c];
    for (int c = 0; c < NC; ++c) {
        if (side == 0) keep[c] = w[c];
        else keep[NC * p + c] = w[NC * p + c];
    }
    for (int r = 1; r <= p; ++r) {
        for (int i = 0; i <= p - r; ++i)
            for (int c = 0; c < NC; ++c) w[NC * i + c] = fmul(fadd(w[NC * i + c], w[NC * (i + 1) + c]), 0.5);
        for (int c = 0; c < NC; ++c) {
            if (side == 0) keep[NC * r + c] = w[c];
            else keep[NC * (p - r) + c] = w[NC * (p - r) + c];
        }
    }
    for (int i = 0; i <= p; ++i)
        for (int c = 0; c < NC; ++c) Q[i * s + c] = keep[NC * i + c];
}

// ------------------------------------------------------- rational pieces
//
// A rational curve is C = A/W, A = sum N_i w_i P_i, W = sum N_i w_i: its
// span's piece is the rational Bezier of the homogeneous points H_j =
// (W_j Q_j, W_j) that the matrix route gives for (w_i P_i, w_i), and its
// halving is the halving of H.  The query tables hold polynomial cubics, so a
// rational node is replaced by its C1 Hermite cubic R and accepted when a
// certified bound of |C - R| meets the tolerance (the paper's method covers
// non-rational splines only; this extends its error-controlled subdivision
// to them).

// R_0 = C(0), R_3 = C(1), R_1 = C(0) + C'(0)/3, R_2 = C(1) - C'(1)/3, with
// C'(0) = p (H_1 - W_1 C(0)) / W_0 and C'(1) = p (W_{p-1} C(1) - H_{p-1}) / W_p
// (the quotient rule at the ends of a rational Bezier; H_j its first three
// coordinates)
template <int MP, class CF>
__host__ __device__ void rhermite(int p, const double* H, double* R, const CF& cf)
{
    const double a = cf.ap_(p);
    const double* h0 = H;
    const double* h1 = H + 4;
    const double* hm = H + 4 * (p - 1);
    const double* hp = H + 4 * p;
    for (int c = 0; c < 3; ++c) {
        const double c0 = fdiv(h0[c], h0[3]), c1 = fdiv(hp[c], hp[3]);
        R[c] = c0;
        R[3 + c] = fadd(c0, fmul(a, fdiv(fsub(h1[c], fmul(h1[3], c0)), h0[3])));
        R[6 + c] = fadd(c1, fmul(a, fdiv(fsub(hm[c], fmul(hm[3], c1)), hp[3])));
        R[9 + c] = c1;
    }
}

// Certified bound of max_u |C(u) - R(u)|^2 over the node: C - R = (A - W R)/W
// with A - W R a polynomial of degree p + 3, whose Bernstein coefficients
// are A's elevated three times minus those of the product W R,
//   (W R)_k = sum_j [C(p, j) C(3, k - j) / C(p + 3, k)] W_j R_{k-j};
// the largest coefficient norm bounds |A - W R| (convex partition of unity)
// and W >= min_j W_j > 0.
// the coefficients rbound2 uses, which depend on the degree alone: computed
// once per span (the same operations as computing them at every node)
template <int MP>
struct RBoundCoef {
    double ea[3][MP + 3], eb[3][MP + 3];  // elevation n -> n + 1, n = p, p + 1, p + 2
    double pc[MP + 4][4];                 // C(p, j) C(3, k - j) / C(p + 3, k), j = k - 3 + jj
};

template <int MP>
__host__ __device__ void rbound_coef(int p, RBoundCoef<MP>& rc)
{
    for (int d = 0; d < 3; ++d) {
        const int n = p + d;
        for (int i = 1; i <= n; ++i) {
            rc.ea[d][i] = fdiv((double)i, (double)(n + 1));
            rc.eb[d][i] = fdiv((double)(n + 1 - i), (double)(n + 1));
        }
    }
    for (int k = 0; k <= p + 3; ++k)
        for (int jj = 0; jj < 4; ++jj) {
            const int j = k - 3 + jj;
            rc.pc[k][jj] = (j >= 0 && j <= p) ? fdiv(fmul(binom_d(p, j), binom_d(3, k - j)), binom_d(p + 3, k)) : 0.0;
        }
}

template <int MP>
__host__ __device__ double rbound2(int p, const double* H, const double* R, const RBoundCoef<MP>& rc)
{
    double e[(MP + 4) * 4], x[(MP + 4) * 4];
    for (int i = 0; i < 4 * (p + 1); ++i) e[i] = H[i];
    for (int n = p; n < p + 3; ++n) {
        for (int c = 0; c < 4; ++c) {
            x[c] = e[c];
            x[4 * (n + 1) + c] = e[4 * n + c];
        }
        for (int i = 1; i <= n; ++i) {
            const double a = rc.ea[n - p][i], b = rc.eb[n - p][i];
            for (int c = 0; c < 4; ++c) x[4 * i + c] = fadd(fmul(a, e[4 * (i - 1) + c]), fmul(b, e[4 * i + c]));
        }
        for (int i = 0; i < 4 * (n + 2); ++i) e[i] = x[i];
    }
    double wmin = H[3];
    for (int j = 1; j <= p; ++j)
        if (H[4 * j + 3] < wmin) wmin = H[4 * j + 3];
    double b = 0.0;
    for (int k = 0; k <= p + 3; ++k) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        const int jlo = k - 3 > 0 ? k - 3 : 0, jhi = k < p ? k : p;
        for (int j = jlo; j <= jhi; ++j) {
            const double cw = fmul(rc.pc[k][j - (k - 3)], H[4 * j + 3]);
            const double* r = R + 3 * (k - j);
            sx = fadd(sx, fmul(cw, r[0]));
            sy = fadd(sy, fmul(cw, r[1]));
            sz = fadd(sz, fmul(cw, r[2]));
        }
        const double dx = fsub(e[4 * k], sx), dy = fsub(e[4 * k + 1], sy), dz = fsub(e[4 * k + 2], sz);
        const double d2 = fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
        if (d2 > b) b = d2;
    }
    return fdiv(b, fmul(wmin, wmin));
}

__host__ __device__ double dyadic_t(double tq, double tq1, int64_t k, int L)
{
    if (k == 0) return tq;
    if (k == ((int64_t)1 << L)) return tq1;
    return fadd(tq, fmul(fsub(tq1, tq), ldexp((double)k, -L)));
}

__host__ __device__ int find_le(const int64_t* __restrict__ off, int64_t n, int64_t x)
{
    // largest i in [0, n) with off[i] <= x
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return (int)lo;
}

// ------------------------------------------------------------- validation

struct DecWS {
    int* err;       // [1] bit 0: invalid data, bit 1: not converged
    int* maxdeg;    // [1]
    int64_t* cnt;   // [n_slots] leaves per slot, then exclusive offsets
    int64_t* gcnt;  // [n+1] groups per spline, then offsets
    int64_t* tmp;   // scan temporaries
};

__host__ __device__ bool knots_ok(int p, const double* U, int64_t nU, int64_t nP)
{
    if (p < 1 || nP < p + 1 || nU != nP + p + 1) return false;
    for (int64_t i = 0; i < nU; ++i) {
        if (!isfinite(U[i])) return false;
        if (i > 0 && U[i] < U[i - 1]) return false;
    }
    return U[p] < U[nP];
}

__host__ __device__ double box_diag_d(const double* P, int64_t np)
{
    double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int64_t i = 0; i < np; ++i)
        for (int c = 0; c < 3; ++c) {
            double v = P[3 * i + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
    double dx = fsub(hi[0], lo[0]), dy = fsub(hi[1], lo[1]), dz = fsub(hi[2], lo[2]);
    return fsqrt(fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz)));
}

// rat [n]: 1 for a rational curve whose weights are not all equal (it takes
// the rational walk), else 0 (equal weights: A/W = sum N_i P_i, the basis
// being a partition of unity, so the curve is the non-rational one); flags
// bit 2 of err when any curve is rational
__global__ void k_validate_curves(bspl_curves C, int64_t n_cp, double* diag, int* err, int* maxdeg, int* rat)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C.n) return;
    if (c == 0 && C.cp_off[C.n] != n_cp) atomicOr(err, 1);
    int p = C.degree[c];
    int64_t nP = C.cp_off[c + 1] - C.cp_off[c], nU = C.knot_off[c + 1] - C.knot_off[c];
    bool ok = p >= 1 && p <= kMaxCurveDegree && knots_ok(p, C.knots + C.knot_off[c], nU, nP);
    const double* P = C.cps + 3 * C.cp_off[c];
    if (ok)
        for (int64_t i = 0; i < 3 * nP; ++i)
            if (!isfinite(P[i])) { ok = false; break; }
    int r = 0;
    if (ok && C.weights) {
        const double* w = C.weights + C.cp_off[c];
        for (int64_t i = 0; i < nP; ++i) {
            if (!(isfinite(w[i]) && w[i] > 0.0)) {
                ok = false;
                break;
            }
            if (w[i] != w[0]) r = 1;
        }
    }
    rat[c] = ok ? r : 0;
    diag[c] = ok ? box_diag_d(P, nP) : __longlong_as_double(0x7ff8000000000000LL);
    if (!ok) atomicOr(err, 1);
    else atomicMax(maxdeg, p);
    if (ok && r) atomicOr(err, 4);
}

__global__ void k_validate_surfaces(bspl_surfaces S, int64_t n_cp, double* diag, int* err, int* maxdeg)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.n) return;
    if (s == 0 && S.cp_off[S.n] != n_cp) atomicOr(err, 1);
    int pu = S.deg_u[s], pv = S.deg_v[s], nu = S.n_u[s], nv = S.n_v[s];
    int64_t np = S.cp_off[s + 1] - S.cp_off[s];
    bool ok = pu >= 1 && pv >= 1 && pu <= kMaxSurfDegree && pv <= kMaxSurfDegree && nu > 0 && nv > 0 &&
              np == (int64_t)nu * nv &&
              knots_ok(pu, S.knots_u + S.knot_u_off[s], S.knot_u_off[s + 1] - S.knot_u_off[s], nu) &&
              knots_ok(pv, S.knots_v + S.knot_v_off[s], S.knot_v_off[s + 1] - S.knot_v_off[s], nv);
    const double* P = S.cps + 3 * S.cp_off[s];
    if (ok)
        for (int64_t i = 0; i < 3 * np; ++i)
            if (!isfinite(P[i])) { ok = false; break; }
    diag[s] = ok ? box_diag_d(P, np) : __longlong_as_double(0x7ff8000000000000LL);
    if (!ok) atomicOr(err, 1);
    else atomicMax(maxdeg, pu > pv ? pu : pv);
}

// ------------------------------------------------------------------ curves

struct CurveLeafOut {
    double* ctrl;
    double* prange;
};

// Walks the subdivision tree of one span depth first.  FILL = false counts
// leaves; FILL = true writes them from index `first`.  The nodes on the path
// to depth kStack - 1 are kept, so a node is one halving of its parent;
// deeper nodes are replayed from the deepest kept ancestor.  Either way a
// node is the same sequence of halvings from the span's Bezier piece.
__host__ __device__ inline void set_flag(int* err, int bit)
{
#ifdef __CUDA_ARCH__
    atomicOr(err, bit);
#else
    *err |= bit;
#endif
}

template <int MP, bool FILL, class CF>
__host__ __device__ int64_t walk_span_curve(int p, const double* __restrict__ U, int q, const double* __restrict__ Pl,
                                            double thr2, int64_t first, CurveLeafOut out, int* err, const CF& cf)
{
    constexpr int kStack = MP == 7 ? 16 : (MP == 15 ? 8 : 4);
    constexpr int W = (MP + 1) * 3;
    double stk[kStack][W], Q[W];
    const int np3 = 3 * (p + 1);
    if constexpr (MP > kMatrixMaxDeg) span_blossom<MP>(p, U, q, Pl, stk[0]);
    else span_bezier<MP>(p, U, q, Pl, 1, stk[0]);
    int L = 0;
    int64_t k = 0, count = 0;
    for (;;) {
        if (L == 0) {
            for (int i = 0; i < np3; ++i) Q[i] = stk[0][i];
        } else if (L < kStack) {
            for (int i = 0; i < np3; ++i) Q[i] = stk[L - 1][i];
            halve_keep<MP>(p, Q, 3, (int)(k & 1));
            for (int i = 0; i < np3; ++i) stk[L][i] = Q[i];
        } else {
            for (int i = 0; i < np3; ++i) Q[i] = stk[kStack - 1][i];
            for (int d = kStack; d <= L; ++d) halve_keep<MP>(p, Q, 3, (int)((k >> (L - d)) & 1));
        }
        double R[12];
        to_cubic<MP>(p, Q, 3, R, 3, cf);
        bool accept = true;
        if (p > 3) accept = bound2_curve<MP>(p, Q, 3, R, 3, cf) <= thr2;
        if (!accept && (L >= kDepthCap || count >= kLeafCap)) {
            accept = true;
            set_flag(err, 2);
        }
        if (accept) {
            if (FILL) {
                int64_t o = first + count;
                double* dst = out.ctrl + 12 * o;
                for (int i = 0; i < 12; ++i) dst[i] = R[i];
                out.prange[2 * o] = dyadic_t(U[q], U[q + 1], k, L);
                out.prange[2 * o + 1] = dyadic_t(U[q], U[q + 1], k + 1, L);
            }
            ++count;
            while (L > 0 && (k & 1)) {
                k >>= 1;
                --L;
            }
            if (L == 0) break;
            k += 1;
        } else {
            ++L;
            k <<= 1;
        }
    }
    return count;
}

// the same walk over the homogeneous piece of a span of a rational curve
// (weights wl of its p + 1 control points), each node replaced by its
// Hermite cubic and accepted by the bound rbound2
template <int MP, bool FILL, class CF>
__host__ __device__ int64_t walk_span_rcurve(int p, const double* __restrict__ U, int q,
                                             const double* __restrict__ Pl, const double* __restrict__ wl,
                                             double thr2, int64_t first, CurveLeafOut out, int* err, const CF& cf)
{
    constexpr int kStack = MP == 7 ? 12 : (MP == 15 ? 6 : 3);
    constexpr int W = (MP + 1) * 4;
    double stk[kStack][W], H[W];
    const int np4 = 4 * (p + 1);
    if constexpr (MP > kMatrixMaxDeg) span_blossom<MP, 4>(p, U, q, Pl, stk[0], wl);
    else span_bezier<MP, 4>(p, U, q, Pl, 1, stk[0], wl);
    RBoundCoef<MP> rc;
    rbound_coef<MP>(p, rc);
    int L = 0;
    int64_t k = 0, count = 0;
    for (;;) {
        if (L == 0) {
            for (int i = 0; i < np4; ++i) H[i] = stk[0][i];
        } else if (L < kStack) {
            for (int i = 0; i < np4; ++i) H[i] = stk[L - 1][i];
            halve_keep<MP, 4>(p, H, 4, (int)(k & 1));
            for (int i = 0; i < np4; ++i) stk[L][i] = H[i];
        } else {
            for (int i = 0; i < np4; ++i) H[i] = stk[kStack - 1][i];
            for (int d = kStack; d <= L; ++d) halve_keep<MP, 4>(p, H, 4, (int)((k >> (L - d)) & 1));
        }
        double R[12];
        rhermite<MP>(p, H, R, cf);
        bool accept = rbound2<MP>(p, H, R, rc) <= thr2;
        if (!accept && (L >= kDepthCap || count >= kLeafCap)) {
            accept = true;
            set_flag(err, 2);
        }
        if (accept) {
            if (FILL) {
                int64_t o = first + count;
                double* dst = out.ctrl + 12 * o;
                for (int i = 0; i < 12; ++i) dst[i] = R[i];
                out.prange[2 * o] = dyadic_t(U[q], U[q + 1], k, L);
                out.prange[2 * o + 1] = dyadic_t(U[q], U[q + 1], k + 1, L);
            }
            ++count;
            while (L > 0 && (k & 1)) {
                k >>= 1;
                --L;
            }
            if (L == 0) break;
            k += 1;
        } else {
            ++L;
            k <<= 1;
        }
    }
    return count;
}

// the walk of one span slot by one thread: slot = cp_off[c] + (q - p); this
// instance handles degrees (MP/2, MP] (1..7, 8..15, 16..31, 32..63) of the
// rational curves (RAT) or of the others; invalid curves carry a NaN
// diagonal and are skipped
template <int MP, bool FILL, bool RAT, class CF>
__device__ __forceinline__ void walk_slot(const bspl_curves& C, const double* __restrict__ diag, double tol_rel,
                                          int64_t n_slots, int64_t* __restrict__ cnt, CurveLeafOut out, int* err,
                                          const int* __restrict__ rat, const CF& cf)
{
    int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    int c = find_le(C.cp_off, C.n, slot);
    int p = C.degree[c];
    constexpr int lo = MP == 7 ? 1 : (MP + 1) / 2;
    if (p < lo || p > MP || !(diag[c] >= 0.0) || (rat[c] != 0) != RAT) return;
    int64_t nP = C.cp_off[c + 1] - C.cp_off[c];
    int q = p + (int)(slot - C.cp_off[c]);
    const double* U = C.knots + C.knot_off[c];
    int64_t r = 0;
    if (q <= nP - 1 && U[q] < U[q + 1]) {
        double thr = fmul(tol_rel, diag[c]);
        if constexpr (RAT)
            r = walk_span_rcurve<MP, FILL>(p, U, q, C.cps + 3 * (C.cp_off[c] + q - p), C.weights + C.cp_off[c] + q - p,
                                           fmul(thr, thr), FILL ? cnt[slot] : 0, out, err, cf);
        else
            r = walk_span_curve<MP, FILL>(p, U, q, C.cps + 3 * (C.cp_off[c] + q - p), fmul(thr, thr),
                                          FILL ? cnt[slot] : 0, out, err, cf);
    }
    if (!FILL) cnt[slot] = r;
}

// slot = cp_off[c] + (q - p), q in [p, ncp-1]; RAT: the rational curves
// (rat[c] = 1) only, else the others
template <int MP, bool FILL, bool RAT = false>
__global__ void k_walk_curves(bspl_curves C, const double* __restrict__ diag, double tol_rel, int64_t n_slots,
                              int64_t* __restrict__ cnt, CurveLeafOut out, int* err, const int* __restrict__ rat)
{
    if constexpr (MP <= kCoefTableMaxDeg) {
        __shared__ RedCoef<MP> cf;  // the block's coefficient tables
        fill_coef<MP>(cf);
        walk_slot<MP, FILL, RAT>(C, diag, tol_rel, n_slots, cnt, out, err, rat, cf);
    } else {
        walk_slot<MP, FILL, RAT>(C, diag, tol_rel, n_slots, cnt, out, err, rat, CoefInline{});
    }
}

// ---------------------------------------------------------------- surfaces

// a net of (degree + 1) x (degree + 1) points, flat: point (a, b) at (a * kSN + b) * 3
constexpr int kSN = kMaxSurfDegree + 1;

// reduce along u for every v column, then along v for every u row
using SurfCoef = RedCoef<kMaxSurfDegree>;

__host__ __device__ void surf_to_bicubic(int pu, int pv, const double* Q, double* R /* [4*4*3] */, const SurfCoef& cf)
{
    double Rp[4 * kSN * 3];
    for (int j = 0; j <= pv; ++j) {
        double col[kSN * 3], r[12];
        for (int i = 0; i <= pu; ++i)
            for (int c = 0; c < 3; ++c) col[3 * i + c] = Q[(i * kSN + j) * 3 + c];
        to_cubic<kMaxSurfDegree>(pu, col, 3, r, 3, cf);
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) Rp[(i * kSN + j) * 3 + c] = r[3 * i + c];
    }
    for (int i = 0; i < 4; ++i) {
        double r[12];
        to_cubic<kMaxSurfDegree>(pv, Rp + i * kSN * 3, 3, r, 3, cf);
        for (int j = 0; j < 4; ++j)
            for (int c = 0; c < 3; ++c) R[(i * 4 + j) * 3 + c] = r[3 * j + c];
    }
}

__host__ __device__ void elevate_to(int from, int to, double* w /* [kSN*3] */, const SurfCoef& cf)
{
    double x[kSN * 3];
    for (int n = from; n < to; ++n) {
        elevate<kMaxSurfDegree>(n, w, x, 3, cf);
        for (int i = 0; i <= n + 1; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = x[3 * i + c];
    }
}

// certified bound at degrees (max(pu,3), max(pv,3)): Q elevated along u then
// v, R elevated along v then u
__host__ __device__ double surf_bound2(int pu, int pv, const double* Q, const double* R, const SurfCoef& cf)
{
    int eu = pu > 3 ? pu : 3, ev = pv > 3 ? pv : 3;
    double Qe[kSN * kSN * 3], Re[kSN * kSN * 3];
    for (int j = 0; j <= pv; ++j) {
        double w[kSN * 3];
        for (int i = 0; i <= pu; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Q[(i * kSN + j) * 3 + c];
        elevate_to(pu, eu, w, cf);
        for (int i = 0; i <= eu; ++i)
            for (int c = 0; c < 3; ++c) Qe[(i * kSN + j) * 3 + c] = w[3 * i + c];
    }
    for (int i = 0; i <= eu; ++i) {
        double w[kSN * 3];
        for (int j = 0; j <= pv; ++j)
            for (int c = 0; c < 3; ++c) w[3 * j + c] = Qe[(i * kSN + j) * 3 + c];
        elevate_to(pv, ev, w, cf);
        for (int j = 0; j <= ev; ++j)
            for (int c = 0; c < 3; ++c) Qe[(i * kSN + j) * 3 + c] = w[3 * j + c];
    }
    for (int i = 0; i < 4; ++i) {
        double w[kSN * 3];
        for (int j = 0; j < 4; ++j)
            for (int c = 0; c < 3; ++c) w[3 * j + c] = R[(i * 4 + j) * 3 + c];
        elevate_to(3, ev, w, cf);
        for (int j = 0; j <= ev; ++j)
            for (int c = 0; c < 3; ++c) Re[(i * kSN + j) * 3 + c] = w[3 * j + c];
    }
    for (int j = 0; j <= ev; ++j) {
        double w[kSN * 3];
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Re[(i * kSN + j) * 3 + c];
        elevate_to(3, eu, w, cf);
        for (int i = 0; i <= eu; ++i)
            for (int c = 0; c < 3; ++c) Re[(i * kSN + j) * 3 + c] = w[3 * i + c];
    }
    double b = 0.0;
    for (int i = 0; i <= eu; ++i)
        for (int j = 0; j <= ev; ++j) {
            const double* a = Qe + (i * kSN + j) * 3;
            const double* r = Re + (i * kSN + j) * 3;
            double dx = fsub(a[0], r[0]), dy = fsub(a[1], r[1]), dz = fsub(a[2], r[2]);
            double e = fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
            if (e > b) b = e;
        }
    return b;
}

// squared certified deviation of the reduction along one direction alone:
// every column (dir 0, along u) or row (dir 1, along v) of the net reduced to
// a cubic and bounded against itself (degree > 3 in that direction)
__host__ __device__ double surf_dir_dev2(int pu, int pv, const double* Q, int dir, const SurfCoef& cf)
{
    double b = 0.0;
    if (dir == 0) {
        for (int j = 0; j <= pv; ++j) {
            double col[kSN * 3], r[12];
            for (int i = 0; i <= pu; ++i)
                for (int c = 0; c < 3; ++c) col[3 * i + c] = Q[(i * kSN + j) * 3 + c];
            to_cubic<kMaxSurfDegree>(pu, col, 3, r, 3, cf);
            const double e = bound2_curve<kMaxSurfDegree>(pu, col, 3, r, 3, cf);
            if (e > b) b = e;
        }
    } else {
        for (int i = 0; i <= pu; ++i) {
            double row[kSN * 3], r[12];
            for (int j = 0; j <= pv; ++j)
                for (int c = 0; c < 3; ++c) row[3 * j + c] = Q[(i * kSN + j) * 3 + c];
            to_cubic<kMaxSurfDegree>(pv, row, 3, r, 3, cf);
            const double e = bound2_curve<kMaxSurfDegree>(pv, row, 3, r, 3, cf);
            if (e > b) b = e;
        }
    }
    return b;
}

// split direction of a net that failed the bound: the reduced direction when
// only one is reduced, else the one whose reduction alone deviates more
// (ties -> u).  (The parameter lengths of a span pair can differ by orders
// of magnitude from where its deviation lies.)
__host__ __device__ int surf_split_dir(int pu, int pv, const double* Q, const SurfCoef& cf)
{
    if (pu > 3 && pv <= 3) return 0;
    if (pv > 3 && pu <= 3) return 1;
    return surf_dir_dev2(pu, pv, Q, 0, cf) >= surf_dir_dev2(pu, pv, Q, 1, cf) ? 0 : 1;
}

__host__ __device__ void surf_halve_keep(int pu, int pv, double* Q, int dir, int side)
{
    if (dir == 0) {
        for (int j = 0; j <= pv; ++j) halve_keep<kMaxSurfDegree>(pu, Q + 3 * j, 3 * kSN, side);
    } else {
        for (int i = 0; i <= pu; ++i) halve_keep<kMaxSurfDegree>(pv, Q + 3 * kSN * i, 3, side);
    }
}

// the float nearest above x (x itself when representable)
__host__ __device__ inline float round_up_f32(double x)
{
#ifdef __CUDA_ARCH__
    return __double2float_ru(x);
#else
    const float f = (float)x;
    return (double)f < x ? nextafterf(f, INFINITY) : f;
#endif
}

// Bernstein -> power coefficients of a degree-n piece in place (stride s doubles)
__host__ __device__ void bern_to_power(int n, double* Q, int s)
{
    double a[kSN * 3];
    for (int k = 0; k <= n; ++k)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int j = 0; j <= k; ++j) {
                double m = binom_d(n, j) * binom_d(n - j, k - j);
                if ((k - j) & 1) m = -m;
                acc += m * Q[j * s + c];
            }
            a[3 * k + c] = acc;
        }
    for (int k = 0; k <= n; ++k)
        for (int c = 0; c < 3; ++c) Q[k * s + c] = a[3 * k + c];
}

struct SurfLeafOut {
    double* ctrl;
    double* prange;
    int64_t* patch_span;
    double* patch_box;
    double* rec64;     // box of the ORIGINAL piece is written here (first 6 entries)
    float* rec32;      // the degrees (pu, pv) go to the two pad entries
    double* span_net;  // original span-pair piece, power basis [8][8][3]
    float* span_net32; // the same in FP32
    float* patch_net32; // original piece over each patch, the patch's own power basis, FP32
};

// x rounded up to FP32 (a bound must not shrink when it is stored)
__host__ __device__ inline float up_f(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

// Bounds of the ORIGINAL piece's derivatives over its patch box, in the
// patch's own parameters (s, t) in [0,1]^2, from the Bernstein net Q of
// degree (pu, pv) that the walk holds for the patch: a derivative of a
// Bezier patch is a Bezier patch whose control points are scaled forward
// differences of Q, and the convex-hull property bounds its length by the
// longest of them.  out[0..4]: |S_s|, |S_t|, |S_ss|, |S_st|, |S_tt|;
// out[6..9]: |S_sss|, |S_sst|, |S_stt|, |S_ttt| (rounded up; out[5] is
// left to the caller).
__host__ __device__ inline void patch_bounds(int pu, int pv, const double* Q, float* out)
{
    double m[9] = { 0, 0, 0, 0, 0, 0, 0, 0, 0 };
    // order-(i, j) forward difference of Q at (a, b), one coordinate
    auto diff = [&](int a, int b, int i, int j, int c) {
        const double bi[4][4] = { { 1, 0, 0, 0 }, { -1, 1, 0, 0 }, { 1, -2, 1, 0 }, { -1, 3, -3, 1 } };
        double acc = 0.0;
        for (int x = 0; x <= i; ++x)
            for (int y = 0; y <= j; ++y) acc += bi[i][x] * bi[j][y] * Q[((a + x) * kSN + (b + y)) * 3 + c];
        return acc;
    };
    // falling factorials p!/(p-k)!
    auto ff = [](int p, int k) {
        double r = 1.0;
        for (int i = 0; i < k; ++i) r *= (double)(p - i);
        return r;
    };
    const int ord[9][2] = { { 1, 0 }, { 0, 1 }, { 2, 0 }, { 1, 1 }, { 0, 2 }, { 0, 0 }, { 3, 0 }, { 2, 1 }, { 1, 2 } };
    for (int k = 0; k < 10; ++k) {
        if (k == 5) continue;
        const int i = k < 9 ? ord[k][0] : 0, j = k < 9 ? ord[k][1] : 3;
        if (i > pu || j > pv) continue;  // that derivative vanishes
        const double f = ff(pu, i) * ff(pv, j);
        double mk = 0.0;
        for (int a = 0; a + i <= pu; ++a)
            for (int b = 0; b + j <= pv; ++b) {
                double w2 = 0.0;
                for (int c = 0; c < 3; ++c) {
                    const double d = f * diff(a, b, i, j, c);
                    w2 += d * d;
                }
                mk = fmax(mk, sqrt(w2));
            }
        if (k < 9) m[k] = mk;
        else m[5] = mk;  // k = 9: (0, 3) stored in m[5] temporarily
    }
    for (int k = 0; k < 5; ++k) out[k] = up_f(m[k] * (1.0 + 1e-12));
    out[6] = up_f(m[6] * (1.0 + 1e-12));
    out[7] = up_f(m[7] * (1.0 + 1e-12));
    out[8] = up_f(m[8] * (1.0 + 1e-12));
    out[9] = up_f(m[5] * (1.0 + 1e-12));
}

// Which edges of a patch the distance function is continuously
// differentiable across (bit 0: s = 0, 1: s = 1, 2: t = 0, 3: t = 1).  An
// edge inside its span pair always is; an edge on a knot line is when that
// knot is inside the parameter domain [K[p], K[n]] (n control points, n + p
// + 1 knots) and its multiplicity is below the degree p (the spline is C1 or
// better there).  Span (p <= q <= n - 1, K[q] < K[q + 1]).
__host__ __device__ inline bool knot_line_smooth(const double* K, int p, int n, double x)
{
    if (!(x > K[p] && x < K[n])) return false;
    int mult = 0;
    for (int k = 0; k <= n + p; ++k) mult += K[k] == x ? 1 : 0;
    return mult < p;
}

__host__ __device__ inline int patch_edge_flags(int pu, int pv, const double* U, int nu, int qu, const double* V,
                                                int nv, int qv, const double* pb)
{
    int f = 0;
    if (pb[0] > 0.0 || knot_line_smooth(U, pu, nu, U[qu])) f |= 1;
    if (pb[1] < 1.0 || knot_line_smooth(U, pu, nu, U[qu + 1])) f |= 2;
    if (pb[2] > 0.0 || knot_line_smooth(V, pv, nv, V[qv])) f |= 4;
    if (pb[3] < 1.0 || knot_line_smooth(V, pv, nv, V[qv + 1])) f |= 8;
    return f;
}

template <bool FILL>
__host__ __device__ int64_t walk_span_surface(int pu, int pv, const double* U, int nu, int qu, const double* V,
                                     int qv, const double* P, int nv, double thr2, int64_t slot, int64_t first,
                                     SurfLeafOut out, int* err, const SurfCoef& cf)
{
    double root[kSN * kSN * 3], Q[kSN * kSN * 3];
    {
        // along u for every v index of the local window, then along v
        double T1[kSN * kSN * 3];
        for (int b = 0; b <= pv; ++b) {
            double out_[kSN * 3];
            span_bezier<kMaxSurfDegree>(pu, U, qu, P + 3 * ((int64_t)(qu - pu) * nv + (qv - pv + b)), nv, out_);
            for (int a = 0; a <= pu; ++a)
                for (int c = 0; c < 3; ++c) T1[(a * kSN + b) * 3 + c] = out_[3 * a + c];
        }
        for (int a = 0; a <= pu; ++a) {
            double out_[kSN * 3];
            span_bezier<kMaxSurfDegree>(pv, V, qv, T1 + a * kSN * 3, 1, out_);
            for (int b = 0; b <= pv; ++b)
                for (int c = 0; c < 3; ++c) root[(a * kSN + b) * 3 + c] = out_[3 * b + c];
        }
    }
    if (FILL) {
        // original span-pair piece in power form for the final Newton steps
        double W[kSN * kSN * 3];
        for (int a = 0; a < kSN; ++a)
            for (int b = 0; b < kSN; ++b)
                for (int c = 0; c < 3; ++c)
                    W[(a * kSN + b) * 3 + c] = (a <= pu && b <= pv) ? root[(a * kSN + b) * 3 + c] : 0.0;
        for (int b = 0; b <= pv; ++b) bern_to_power(pu, W + 3 * b, 3 * kSN);
        for (int a = 0; a <= pu; ++a) bern_to_power(pv, W + 3 * kSN * a, 3);
        double* dst = out.span_net + (int64_t)BSPL_SPAN_NET * slot;
        float* dst32 = out.span_net32 + (int64_t)BSPL_SPAN_NET * slot;
        for (int i = 0; i < kSN * kSN * 3; ++i) {
            dst[i] = W[i];
            dst32[i] = (float)W[i];
        }
    }
    int L = 0;
    uint64_t bits = 0;  // path bits, most recent in bit 0
    uint64_t dirs = 0;  // bit l: the direction the ancestor at depth l was split in
    int64_t count = 0;
    for (;;) {
        // replay the path from the root
        for (int i = 0; i < kSN * kSN * 3; ++i) Q[i] = root[i];
        int Lu = 0, Lv = 0;
        int64_t ku = 0, kv = 0;
        for (int l = 0; l < L; ++l) {
            int side = (int)((bits >> (L - 1 - l)) & 1);
            int dir = (int)((dirs >> l) & 1);
            surf_halve_keep(pu, pv, Q, dir, side);
            if (dir == 0) {
                ++Lu;
                ku = 2 * ku + side;
            } else {
                ++Lv;
                kv = 2 * kv + side;
            }
        }
        double R[4 * 4 * 3];
        surf_to_bicubic(pu, pv, Q, R, cf);
        bool accept = true;
        if (pu > 3 || pv > 3) accept = surf_bound2(pu, pv, Q, R, cf) <= thr2;
        if (!accept && (Lu + Lv >= kDepthCap || count >= kLeafCap)) {
            accept = true;
            set_flag(err, 2);
        }
        if (accept) {
            if (FILL) {
                int64_t o = first + count;
                double* dst = out.ctrl + 48 * o;
                for (int i = 0; i < 48; ++i) dst[i] = R[i];
                double* pr = out.prange + 4 * o;
                pr[0] = dyadic_t(U[qu], U[qu + 1], ku, Lu);
                pr[1] = dyadic_t(U[qu], U[qu + 1], ku + 1, Lu);
                pr[2] = dyadic_t(V[qv], V[qv + 1], kv, Lv);
                pr[3] = dyadic_t(V[qv], V[qv + 1], kv + 1, Lv);
                out.patch_span[o] = slot;
                double* pb = out.patch_box + 4 * o;
                pb[0] = ldexp((double)ku, -Lu);
                pb[1] = ldexp((double)(ku + 1), -Lu);
                pb[2] = ldexp((double)kv, -Lv);
                pb[3] = ldexp((double)(kv + 1), -Lv);
                // box of the original piece (conservative for the original surface)
                double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
                for (int a = 0; a <= pu; ++a)
                    for (int b = 0; b <= pv; ++b)
                        for (int c = 0; c < 3; ++c) {
                            lo[c] = fmin(lo[c], Q[(a * kSN + b) * 3 + c]);
                            hi[c] = fmax(hi[c], Q[(a * kSN + b) * 3 + c]);
                        }
                double* rb = out.rec64 + (int64_t)BSPL_SREC64 * o;
                for (int c = 0; c < 3; ++c) {
                    rb[c] = lo[c];
                    rb[3 + c] = hi[c];
                }
                float* rf = out.rec32 + (int64_t)BSPL_SREC32 * o;
                rf[54] = (float)pu;
                rf[55] = (float)pv;
                // the original piece over the patch in its own power basis
                {
                    double W[kSN * kSN * 3];
                    for (int a = 0; a < kSN; ++a)
                        for (int b = 0; b < kSN; ++b)
                            for (int c = 0; c < 3; ++c)
                                W[(a * kSN + b) * 3 + c] = (a <= pu && b <= pv) ? Q[(a * kSN + b) * 3 + c] : 0.0;
                    for (int b = 0; b <= pv; ++b) bern_to_power(pu, W + 3 * b, 3 * kSN);
                    for (int a = 0; a <= pu; ++a) bern_to_power(pv, W + 3 * kSN * a, 3);
                    float* pn = out.patch_net32 + (int64_t)BSPL_SPAN_NET * o;
                    for (int i = 0; i < kSN * kSN * 3; ++i) pn[i] = (float)W[i];
                    // the weighted L1 norms of those FP32 coefficients that
                    // bound the rounding of their Horner evaluation (weights
                    // 1, i, j, i(i-1), ij, j(j-1) of the term s^i t^j),
                    // without the constant term (the query's), rounded up
                    double L[6] = { 0.0, 0.0, 0.0, 0.0, 0.0, 0.0 };
                    for (int a = 0; a <= pu; ++a)
                        for (int b = 0; b <= pv; ++b) {
                            if ((a | b) == 0) continue;
                            double x = 0.0;
                            for (int c = 0; c < 3; ++c) x += fabs((double)pn[(a * kSN + b) * 3 + c]);
                            L[0] += x;
                            L[1] += a * x;
                            L[2] += b * x;
                            L[3] += a * (a - 1) * x;
                            L[4] += a * b * x;
                            L[5] += b * (b - 1) * x;
                        }
                    for (int k = 0; k < 6; ++k) rf[66 + k] = round_up_f32(L[k]);
                }
                patch_bounds(pu, pv, Q, rf + 56);
                rf[61] = (float)patch_edge_flags(pu, pv, U, nu, qu, V, nv, qv, pb);
            }
            ++count;
            while (L > 0 && (bits & 1)) {
                bits >>= 1;
                --L;
            }
            if (L == 0) break;
            bits |= 1;
        } else {
            const int dir = surf_split_dir(pu, pv, Q, cf);
            dirs = (dirs & ~(1ull << L)) | ((uint64_t)dir << L);
            ++L;
            bits <<= 1;
        }
    }
    return count;
}

// slot = cp_off[s] + a * n_v + b, a = qu - pu, b = qv - pv
template <bool FILL>
__global__ void k_walk_surfaces(bspl_surfaces S, const double* __restrict__ diag, double tol_rel,
                                int64_t n_slots, int64_t* __restrict__ cnt, SurfLeafOut out, int* err)
{
    __shared__ SurfCoef cf;
    fill_coef<kMaxSurfDegree>(cf);
    int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    int s = find_le(S.cp_off, S.n, slot);
    if (!(diag[s] >= 0.0)) return;  // invalid surface
    int pu = S.deg_u[s], pv = S.deg_v[s], nu = S.n_u[s], nv = S.n_v[s];
    int64_t loc = slot - S.cp_off[s];
    int a = (int)(loc / nv), b = (int)(loc % nv);
    int qu = pu + a, qv = pv + b;
    const double* U = S.knots_u + S.knot_u_off[s];
    const double* V = S.knots_v + S.knot_v_off[s];
    int64_t r = 0;
    if (qu <= nu - 1 && qv <= nv - 1 && U[qu] < U[qu + 1] && V[qv] < V[qv + 1]) {
        double thr = fmul(tol_rel, diag[s]);
        r = walk_span_surface<FILL>(pu, pv, U, nu, qu, V, qv, S.cps + 3 * S.cp_off[s], nv, fmul(thr, thr), slot,
                                    FILL ? cnt[slot] : 0, out, err, cf);
    }
    if (!FILL) cnt[slot] = r;
}

// --------------------------------------------------------------- tables

__device__ float down32(double x) { return __double2float_rd(x); }
__device__ float up32(double x) { return __double2float_ru(x); }

// curve segment records: box of the cubic's control points, power basis
// a0 + a1 u + a2 u^2 + a3 u^3 = [1 u u^2 u^3] B_3 R
__global__ void k_curve_records(const double* __restrict__ ctrl, int64_t nseg, double* __restrict__ rec64,
                                float* __restrict__ rec32)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const double* R = ctrl + 12 * s;
    double* o = rec64 + (int64_t)BSPL_CREC64 * s;
    float* f = rec32 + (int64_t)BSPL_CREC32 * s;
    for (int c = 0; c < 3; ++c) {
        double r0 = R[c], r1 = R[3 + c], r2 = R[6 + c], r3 = R[9 + c];
        double lo = fmin(fmin(r0, r1), fmin(r2, r3)), hi = fmax(fmax(r0, r1), fmax(r2, r3));
        double a0 = r0, a1 = 3.0 * (r1 - r0), a2 = 3.0 * (r0 - 2.0 * r1 + r2), a3 = (r3 - r0) + 3.0 * (r1 - r2);
        o[c] = lo;
        o[3 + c] = hi;
        o[6 + c] = a0;
        o[9 + c] = a1;
        o[12 + c] = a2;
        o[15 + c] = a3;
        f[c] = down32(lo);
        f[3 + c] = up32(hi);
        f[6 + c] = (float)a0;
        f[9 + c] = (float)a1;
        f[12 + c] = (float)a2;
        f[15 + c] = (float)a3;
        f[18 + c] = (float)(a0 - (double)f[6 + c]);  // a0 = f[6 + c] + f[18 + c] to ~2^-48 relative
        f[21 + c] = 0.f;
    }
}

// patch records: box already written (original piece); power basis of the
// bicubic a[i][j] (i: u power, j: v power) = B_3 R B_3^T
__global__ void k_patch_records(const double* __restrict__ ctrl, int64_t nseg, double* __restrict__ rec64,
                                float* __restrict__ rec32)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const double* R = ctrl + 48 * s;
    double* o = rec64 + (int64_t)BSPL_SREC64 * s;
    float* f = rec32 + (int64_t)BSPL_SREC32 * s;
    const double M[4][4] = { { 1, 0, 0, 0 }, { -3, 3, 0, 0 }, { 3, -6, 3, 0 }, { -1, 3, -3, 1 } };
    for (int c = 0; c < 3; ++c) {
        double T[4][4];
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) acc += M[i][k] * R[(k * 4 + j) * 3 + c];
                T[i][j] = acc;
            }
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) acc += T[i][k] * M[j][k];
                o[6 + (i * 4 + j) * 3 + c] = acc;
                f[6 + (i * 4 + j) * 3 + c] = (float)acc;
            }
        f[c] = down32(o[c]);
        f[3 + c] = up32(o[3 + c]);
    }
    // f[54], f[55] hold the span-pair degrees, written by the filling walk
}

// group records: union box of up to BSPL_GROUP consecutive segments of one
// spline and a point on the piece (the first control point of its first segment)
__global__ void k_group_records(const int64_t* __restrict__ seg_off, const int64_t* __restrict__ grp_off, int64_t n,
                                int64_t n_grp, const double* __restrict__ rec64, int rec_w,
                                const double* __restrict__ ctrl, int ctrl_w, double* __restrict__ grp64,
                                float* __restrict__ grp32)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_grp) return;
    int c = find_le(grp_off, n, g);
    while (c + 1 < n && grp_off[c + 1] <= g) ++c;
    int64_t s0 = seg_off[c] + (g - grp_off[c]) * BSPL_GROUP;
    int64_t s1 = min(s0 + BSPL_GROUP, seg_off[c + 1]);
    double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int64_t s = s0; s < s1; ++s)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], rec64[(int64_t)rec_w * s + k]);
            hi[k] = fmax(hi[k], rec64[(int64_t)rec_w * s + 3 + k]);
        }
    double* o = grp64 + (int64_t)BSPL_GREC64 * g;
    float* f = grp32 + (int64_t)BSPL_GREC32 * g;
    for (int k = 0; k < 3; ++k) {
        o[k] = lo[k];
        o[3 + k] = hi[k];
        o[6 + k] = ctrl[(int64_t)ctrl_w * s0 + k];
        o[9 + k] = 0.0;
        f[k] = down32(lo[k]);
        f[3 + k] = up32(hi[k]);
        f[6 + k] = (float)o[6 + k];
        f[9 + k] = 0.f;
    }
}

// seg_off[c] = offset of the spline's first slot; group counts per spline
__global__ void k_seg_off(const int64_t* __restrict__ cp_off, int64_t n, const int64_t* __restrict__ off,
                          int64_t n_cp, int64_t* __restrict__ seg_off, int64_t* __restrict__ gcnt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n) return;
    int64_t tot = off[n_cp];
    int64_t v = c < n ? off[cp_off[c]] : tot;
    seg_off[c] = v;
    if (c < n) {
        int64_t v1 = (c + 1 < n) ? off[cp_off[c + 1]] : tot;
        gcnt[c] = (v1 - v + BSPL_GROUP - 1) / BSPL_GROUP;
    } else {
        gcnt[c] = 0;
    }
}

__global__ void k_totals(const int64_t* __restrict__ off, int64_t n_cp, const int64_t* __restrict__ goff, int64_t n,
                         const int* __restrict__ flags, int64_t* __restrict__ dst)
{
    dst[0] = off[n_cp];
    dst[1] = goff[n];
    dst[2] = flags[0];
}

__global__ void k_copy_i64(const int64_t* __restrict__ a, int64_t* __restrict__ b, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

template <class K, class... A>
void launch1d(K kernel, int64_t n, cudaStream_t s, A... args)
{
    if (n <= 0) return;
    int th = 128;
    kernel<<<ceil_div(n, th), th, 0, s>>>(args...);
}

}  // namespace

// the walks of every span of the curve set: one launch per degree class
// (1-7, 8-15, 16-31, 32-63) present, for the non-rational curves and, when
// there are any, for the rational ones
template <bool FILL>
void walk_curves(const bspl_curves& C, const double* diag, double tol_rel, int64_t n_cp, int64_t* cnt,
                 CurveLeafOut o, int* err, const int* rat, int maxdeg, bool any_rat, cudaStream_t s)
{
    launch1d(k_walk_curves<7, FILL>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 7) launch1d(k_walk_curves<15, FILL>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 15) launch1d(k_walk_curves<31, FILL>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 31) launch1d(k_walk_curves<63, FILL>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (!any_rat) return;
    launch1d(k_walk_curves<7, FILL, true>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 7) launch1d(k_walk_curves<15, FILL, true>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 15) launch1d(k_walk_curves<31, FILL, true>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
    if (maxdeg > 31) launch1d(k_walk_curves<63, FILL, true>, n_cp, s, C, diag, tol_rel, n_cp, cnt, o, err, rat);
}

size_t decompose_ws_bytes(int is_surface, int64_t n, int64_t n_cp_total)
{
    (void)is_surface;
    Carver cv(nullptr, 0);
    cv.take<int>(4);
    cv.take<int64_t>((size_t)n_cp_total + 1);
    cv.take<int64_t>((size_t)n + 1);
    cv.take<int64_t>(scan_tmp_elems(n_cp_total + 1) + scan_tmp_elems(n + 1));
    cv.take<int64_t>(4);
    cv.take<int>((size_t)n);
    return cv.used + 256;
}

#define CK(x)                                      \
    do {                                           \
        if ((x) != cudaSuccess) return BSPL_ECUDA; \
    } while (0)

static bspl_status decompose_impl(int is_surface, const void* splines, double tol_rel, bspl_segments* out,
                                  int64_t* total, void* ws, size_t ws_bytes, cudaStream_t s)
{
    const bspl_curves* CC = (const bspl_curves*)splines;
    const bspl_surfaces* SS = (const bspl_surfaces*)splines;
    if (!splines || !out || !total) return BSPL_EINVAL;
    int64_t n = is_surface ? SS->n : CC->n;
    int64_t n_cp = out->n_cp_total;
    const int64_t* cp_off = is_surface ? SS->cp_off : CC->cp_off;
    if (n <= 0 || n_cp <= 0 || !out->seg_off || !out->diag || !cp_off) return BSPL_EINVAL;
    if (!(tol_rel >= 0.0) || !(tol_rel < INFINITY)) return BSPL_EINVAL;
    if (!ws || ws_bytes < decompose_ws_bytes(is_surface, n, n_cp)) return BSPL_EINVAL;
    Carver cv(ws, ws_bytes);
    DecWS w;
    int* flags = cv.take<int>(4);
    w.err = flags;
    w.maxdeg = flags + 1;
    w.cnt = cv.take<int64_t>((size_t)n_cp + 1);
    w.gcnt = cv.take<int64_t>((size_t)n + 1);
    w.tmp = cv.take<int64_t>(scan_tmp_elems(n_cp + 1) + scan_tmp_elems(n + 1));
    int64_t* dev_tot = cv.take<int64_t>(4);
    int* rat = cv.take<int>((size_t)n);
    CK(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    CK(cudaMemsetAsync(w.cnt, 0, sizeof(int64_t) * (size_t)(n_cp + 1), s));

    // validation (invalid splines get a NaN diagonal, which the walks skip,
    // and raise bit 0)
    if (is_surface) launch1d(k_validate_surfaces, n, s, *SS, n_cp, out->diag, w.err, w.maxdeg);
    else launch1d(k_validate_curves, n, s, *CC, n_cp, out->diag, w.err, w.maxdeg, rat);
    CK(cudaGetLastError());
    int hf[2];
    CK(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hf[0] & 1) return BSPL_EINVAL;
    const int maxdeg = hf[1];
    const bool any_rat = (hf[0] & 4) != 0;

    // counting pass
    if (is_surface) {
        SurfLeafOut o{};
        launch1d(k_walk_surfaces<false>, n_cp, s, *SS, (const double*)out->diag, tol_rel, n_cp, w.cnt, o,
                 w.err);
    } else {
        CurveLeafOut o{};
        walk_curves<false>(*CC, out->diag, tol_rel, n_cp, w.cnt, o, w.err, rat, maxdeg, any_rat, s);
    }
    CK(cudaGetLastError());
    CK(exclusive_scan_i64(w.cnt, w.cnt, n_cp + 1, w.tmp, s));
    launch1d(k_seg_off, n + 1, s, cp_off, n, (const int64_t*)w.cnt, n_cp, out->seg_off, w.gcnt);
    CK(cudaGetLastError());
    CK(exclusive_scan_i64(w.gcnt, w.gcnt, n + 1, w.tmp + scan_tmp_elems(n_cp + 1), s));
    k_totals<<<1, 1, 0, s>>>(w.cnt, n_cp, w.gcnt, n, flags, dev_tot);
    CK(cudaGetLastError());
    int64_t h[3];
    CK(cudaMemcpyAsync(h, dev_tot, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *total = h[0];
    int64_t n_grp = h[1];
    int err = (int)h[2];
    if (out->grp_off) launch1d(k_copy_i64, n + 1, s, (const int64_t*)w.gcnt, out->grp_off, n + 1);
    if (out->ctrl == nullptr) {
        CK(cudaGetLastError());
        return (err & 2) ? BSPL_ENOTCONV : BSPL_OK;
    }
    if (h[0] > out->capacity || n_grp > out->grp_capacity) return BSPL_ENOSPACE;
    if (!out->prange || !out->rec64 || !out->rec32 || !out->grp_off || !out->grp64 || !out->grp32)
        return BSPL_EINVAL;
    if (is_surface && (!out->patch_span || !out->patch_box || !out->span_net || !out->span_net32 ||
                       !out->patch_net32))
        return BSPL_EINVAL;
    out->is_surface = is_surface;
    out->n = n;
    out->tol_rel = tol_rel;

    // splines ranked by descending piece count (stable: ties by index), for
    // the heaviest-first order of the query calls' work-stealing launches
    if (out->spline_rank) {
        std::vector<int64_t> off((size_t)n + 1);
        CK(cudaMemcpyAsync(off.data(), out->seg_off, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<int32_t> idx((size_t)n), rank((size_t)n);
        for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = (int32_t)i;
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
            return off[(size_t)a + 1] - off[(size_t)a] > off[(size_t)b + 1] - off[(size_t)b];
        });
        for (int64_t r = 0; r < n; ++r) rank[(size_t)idx[(size_t)r]] = (int32_t)r;
        CK(cudaMemcpyAsync(out->spline_rank, rank.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }

    // filling pass and query tables
    if (is_surface) {
        SurfLeafOut o{ out->ctrl, out->prange, out->patch_span, out->patch_box, out->rec64, out->rec32,
                       out->span_net, out->span_net32, out->patch_net32 };
        launch1d(k_walk_surfaces<true>, n_cp, s, *SS, (const double*)out->diag, tol_rel, n_cp, w.cnt, o, w.err);
        launch1d(k_patch_records, h[0], s, (const double*)out->ctrl, h[0], out->rec64, out->rec32);
        launch1d(k_group_records, n_grp, s, (const int64_t*)out->seg_off, (const int64_t*)out->grp_off, n, n_grp,
                 (const double*)out->rec64, (int)BSPL_SREC64, (const double*)out->ctrl, 48, out->grp64,
                 out->grp32);
    } else {
        CurveLeafOut o{ out->ctrl, out->prange };
        walk_curves<true>(*CC, out->diag, tol_rel, n_cp, w.cnt, o, w.err, rat, maxdeg, any_rat, s);
        launch1d(k_curve_records, h[0], s, (const double*)out->ctrl, h[0], out->rec64, out->rec32);
        launch1d(k_group_records, n_grp, s, (const int64_t*)out->seg_off, (const int64_t*)out->grp_off, n, n_grp,
                 (const double*)out->rec64, (int)BSPL_CREC64, (const double*)out->ctrl, 12, out->grp64,
                 out->grp32);
    }
    CK(cudaGetLastError());
    return (err & 2) ? BSPL_ENOTCONV : BSPL_OK;
}

bspl_status decompose_curves(const bspl_curves* c, double tol_rel, bspl_segments* out, int64_t* total, void* ws,
                             size_t ws_bytes, cudaStream_t s)
{
    return decompose_impl(0, c, tol_rel, out, total, ws, ws_bytes, s);
}

bspl_status decompose_surfaces(const bspl_surfaces* c, double tol_rel, bspl_segments* out, int64_t* total,
                               void* ws, size_t ws_bytes, cudaStream_t s)
{
    return decompose_impl(1, c, tol_rel, out, total, ws, ws_bytes, s);
}

}  // namespace bspl
