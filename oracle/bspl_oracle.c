/*
 * bspl_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of what the GPU
 * library computes, written from the paper (Wu & Zou, "Matrix representation
 * and GPU-optimized parallel B-spline computing", arXiv 2504.11498):
 *
 *   - B-spline evaluation by the Cox-de Boor recursion (Sec. 3, Eq. bsplinebasis)
 *     with basis derivatives (textbook derivative formula).
 *   - Textbook Boehm knot insertion to Bezier segments (cross-check of Sec. 4.2.1).
 *   - The paper's span-wise matrix decomposition Q = B_p^{-1} M A P
 *     (Sec. 4.2.1, Eq. decomfinal), built in the local parameter u.
 *   - Degree elevation (p < 3), the G1-continuous L2-optimal reduction to a cubic
 *     (Sec. 4.2.2, Eqs. G1-condition, epsl, differentiatedelta0/1), a certified
 *     deviation bound and midpoint subdivision until the bound meets the tolerance.
 *   - Projection / inversion (Sec. 3, Eqs. projection, projections, inversion)
 *     ON THE ORIGINAL SPLINE by dense sampling plus safeguarded Newton on
 *     E = D' (Eqs. Dt, Et, E't).
 *   - Tensor-product surface versions of all of the above.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load this library.  It shares no code with the CUDA path.
 *
 * Decomposition decisions (accept a cubic or subdivide) are made in IEEE FP64
 * with a fixed operation order and no FMA contraction (build with
 * -ffp-contract=off).  The CUDA library follows the same arithmetic sequence
 * in code of its own so that segment counts agree bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OMAXP 63          /* highest supported curve degree */
#define OMATP 7           /* highest degree extracted by the matrix route: its
                             FP64 error grows about tenfold every two degrees
                             (6e-14 at 7, 2e-10 at 15, 1e-2 at 31, measured
                             against knot insertion); above it the blossom */
#define ONP (OMAXP + 1)   /* control points of one span */
#define ODEPTH 40         /* subdivision depth cap */
#define OLEAFCAP 65536    /* leaves per span (pair) after which every node is accepted */

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOSPACE = 2, ORC_ENOTCONV = 4 };

/* ------------------------------------------------------------------ */
/* small exact helpers                                                 */
/* ------------------------------------------------------------------ */

/* binomial coefficient, exact in double for the sizes used here (n <= 62) */
static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* Gram entry g_ij = int_0^1 B_i^m B_j^n dt  (Eq. gram) */
double orc_gram(int m, int n, int i, int j)
{
    double num = binom(m, i) * binom(n, j);
    double den = (double)(m + n + 1) * binom(m + n, i + j);
    return num / den;
}

/* ------------------------------------------------------------------ */
/* Cox-de Boor basis (Sec. 3, Eq. bsplinebasis)                          */
/* ------------------------------------------------------------------ */

/* N[j] = N_{q-p+j,p}(t), j = 0..p, for t in span q.  0/0 terms are 0. */
static void cdb_basis(const double* U, int q, int p, double t, double* N)
{
    double cur[ONP + 1], nxt[ONP + 1];
    cur[0] = 1.0; /* N_{q,0} */
    for (int k = 1; k <= p; ++k) {
        for (int j = 0; j <= k; ++j) {
            int i = q - k + j;
            double v = 0.0;
            if (j >= 1) { /* (t - t_i)/(t_{i+k} - t_i) N_{i,k-1} */
                double den = U[i + k] - U[i];
                if (den != 0.0) v += (t - U[i]) / den * cur[j - 1];
            }
            if (j <= k - 1) { /* (t_{i+k+1} - t)/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1} */
                double den = U[i + k + 1] - U[i + 1];
                if (den != 0.0) v += (U[i + k + 1] - t) / den * cur[j];
            }
            nxt[j] = v;
        }
        memcpy(cur, nxt, sizeof(double) * (size_t)(k + 1));
    }
    memcpy(N, cur, sizeof(double) * (size_t)(p + 1));
}

/* values, first and second derivatives of N_{q-p..q,p} at t (textbook rule
 * N'_{i,p} = p N_{i,p-1}/(t_{i+p}-t_i) - p N_{i+1,p-1}/(t_{i+p+1}-t_{i+1})) */
static void cdb_basis_ders(const double* U, int q, int p, double t,
                           double* N0, double* N1, double* N2)
{
    cdb_basis(U, q, p, t, N0);
    for (int j = 0; j <= p; ++j) { N1[j] = 0.0; N2[j] = 0.0; }
    if (p >= 1) {
        double Nm1[ONP + 1];
        cdb_basis(U, q, p - 1, t, Nm1); /* N_{q-p+1+j,p-1} */
        for (int j = 0; j <= p; ++j) {
            int i = q - p + j;
            double v = 0.0;
            if (j >= 1) { double den = U[i + p] - U[i]; if (den != 0.0) v += p * Nm1[j - 1] / den; }
            if (j <= p - 1) { double den = U[i + p + 1] - U[i + 1]; if (den != 0.0) v -= p * Nm1[j] / den; }
            N1[j] = v;
        }
    }
    if (p >= 2) {
        double Nm2[ONP + 1], D1[ONP + 1];
        cdb_basis(U, q, p - 2, t, Nm2); /* N_{q-p+2+j,p-2} */
        for (int j = 0; j <= p - 1; ++j) { /* d/dt N_{q-p+1+j,p-1} */
            int i = q - (p - 1) + j;
            double v = 0.0;
            if (j >= 1) { double den = U[i + p - 1] - U[i]; if (den != 0.0) v += (p - 1) * Nm2[j - 1] / den; }
            if (j <= p - 2) { double den = U[i + p] - U[i + 1]; if (den != 0.0) v -= (p - 1) * Nm2[j] / den; }
            D1[j] = v;
        }
        for (int j = 0; j <= p; ++j) {
            int i = q - p + j;
            double v = 0.0;
            if (j >= 1) { double den = U[i + p] - U[i]; if (den != 0.0) v += p * D1[j - 1] / den; }
            if (j <= p - 1) { double den = U[i + p + 1] - U[i + 1]; if (den != 0.0) v -= p * D1[j] / den; }
            N2[j] = v;
        }
    }
}

/* span q in [p, m] with U[q] <= t < U[q+1]; the closed end maps to the last
 * non-empty span.  m = number of control points - 1. */
static int find_span(const double* U, int m, int p, double t)
{
    int first = -1, last = -1;
    for (int q = p; q <= m; ++q)
        if (U[q] < U[q + 1]) { if (first < 0) first = q; last = q; }
    if (first < 0) return -1;
    if (t <= U[first]) return first;
    if (t >= U[last + 1]) return last;
    for (int q = first; q <= last; ++q)
        if (U[q] <= t && t < U[q + 1]) return q;
    return last;
}

/* exported for the partition-of-unity pin */
int orc_basis(int p, const double* U, int64_t nU, double t, int* span, double* N)
{
    int m = (int)nU - p - 2;
    int q = find_span(U, m, p, t);
    if (q < 0) return ORC_EINVAL;
    *span = q;
    cdb_basis(U, q, p, t, N);
    return ORC_OK;
}

/* C(t), C'(t), C''(t) of a curve (P is [m+1][3]).  w: NULL for a
 * non-rational curve, else the positive weights [m+1] of a rational one
 * (NURBS): C = A/W with A = sum N_i w_i P_i and W = sum N_i w_i, whose
 * derivatives follow from the quotient rule,
 *   C' = (A' - W' C)/W,   C'' = (A'' - 2 W' C' - W'' C)/W. */
static void curve_eval(int p, const double* U, int m, const double* P, const double* w, double t,
                       double* C, double* C1, double* C2)
{
    double N0[ONP + 1], N1[ONP + 1], N2[ONP + 1];
    int q = find_span(U, m, p, t);
    cdb_basis_ders(U, q, p, t, N0, N1, N2);
    for (int c = 0; c < 3; ++c) { C[c] = 0.0; C1[c] = 0.0; C2[c] = 0.0; }
    if (!w) {
        for (int j = 0; j <= p; ++j) {
            const double* Pi = P + 3 * (q - p + j);
            for (int c = 0; c < 3; ++c) {
                C[c] += N0[j] * Pi[c];
                C1[c] += N1[j] * Pi[c];
                C2[c] += N2[j] * Pi[c];
            }
        }
        return;
    }
    double A0[3] = { 0, 0, 0 }, A1[3] = { 0, 0, 0 }, A2[3] = { 0, 0, 0 }, W0 = 0.0, W1 = 0.0, W2 = 0.0;
    for (int j = 0; j <= p; ++j) {
        const double* Pi = P + 3 * (q - p + j);
        double wi = w[q - p + j];
        W0 += N0[j] * wi;
        W1 += N1[j] * wi;
        W2 += N2[j] * wi;
        for (int c = 0; c < 3; ++c) {
            A0[c] += N0[j] * wi * Pi[c];
            A1[c] += N1[j] * wi * Pi[c];
            A2[c] += N2[j] * wi * Pi[c];
        }
    }
    for (int c = 0; c < 3; ++c) {
        C[c] = A0[c] / W0;
        C1[c] = (A1[c] - W1 * C[c]) / W0;
        C2[c] = (A2[c] - 2.0 * W1 * C1[c] - W2 * C[c]) / W0;
    }
}

/* surface S(u,v) with partials; P is [nu][nv][3] row-major, index i along u.
 * wt: NULL for a non-rational surface, else the positive weights [nu][nv]
 * of a rational one: S = A/W with A, W the sums over (w P, w), and the
 * quotient rule
 *   S_u  = (A_u - W_u S)/W,                 S_v  = (A_v - W_v S)/W,
 *   S_uu = (A_uu - 2 W_u S_u - W_uu S)/W,   S_vv = (A_vv - 2 W_v S_v - W_vv S)/W,
 *   S_uv = (A_uv - W_u S_v - W_v S_u - W_uv S)/W. */
static void surface_eval(int pu, int pv, const double* U, int mu, const double* V, int mv,
                         const double* P, const double* wt, int nv, double u, double v, double* out /* [6][3]:
                         S, Su, Sv, Suu, Suv, Svv */)
{
    double Nu0[ONP + 1], Nu1[ONP + 1], Nu2[ONP + 1];
    double Nv0[ONP + 1], Nv1[ONP + 1], Nv2[ONP + 1];
    int qu = find_span(U, mu, pu, u), qv = find_span(V, mv, pv, v);
    cdb_basis_ders(U, qu, pu, u, Nu0, Nu1, Nu2);
    cdb_basis_ders(V, qv, pv, v, Nv0, Nv1, Nv2);
    double A[18], W[6];
    for (int k = 0; k < 18; ++k) A[k] = 0.0;
    for (int k = 0; k < 6; ++k) W[k] = 0.0;
    for (int a = 0; a <= pu; ++a) {
        for (int b = 0; b <= pv; ++b) {
            int64_t ij = (int64_t)(qu - pu + a) * nv + (qv - pv + b);
            const double* Pij = P + 3 * ij;
            double wij = wt ? wt[ij] : 1.0;
            double w[6] = { Nu0[a] * Nv0[b], Nu1[a] * Nv0[b], Nu0[a] * Nv1[b],
                            Nu2[a] * Nv0[b], Nu1[a] * Nv1[b], Nu0[a] * Nv2[b] };
            for (int k = 0; k < 6; ++k) {
                for (int c = 0; c < 3; ++c) A[3 * k + c] += wt ? w[k] * wij * Pij[c] : w[k] * Pij[c];
                W[k] += w[k] * wij;
            }
        }
    }
    if (!wt) {
        memcpy(out, A, sizeof(A));
        return;
    }
    for (int c = 0; c < 3; ++c) {
        double S = A[c] / W[0];
        double Su = (A[3 + c] - W[1] * S) / W[0];
        double Sv = (A[6 + c] - W[2] * S) / W[0];
        out[c] = S;
        out[3 + c] = Su;
        out[6 + c] = Sv;
        out[9 + c] = (A[9 + c] - 2.0 * W[1] * Su - W[3] * S) / W[0];
        out[12 + c] = (A[12 + c] - W[1] * Sv - W[2] * Su - W[4] * S) / W[0];
        out[15 + c] = (A[15 + c] - 2.0 * W[2] * Sv - W[5] * S) / W[0];
    }
}

/* ------------------------------------------------------------------ */
/* batch evaluation                                                     */
/* ------------------------------------------------------------------ */

/* w: NULL (non-rational) or the weights [coff[n]] of every control point */
int orc_eval_curves(int64_t n, const int32_t* deg, const int64_t* koff, const double* knots,
                    const int64_t* coff, const double* cps, const double* w, int64_t nq, const int32_t* qc,
                    const double* t, double* out /* [nq][3][3] */)
{
    for (int64_t k = 0; k < nq; ++k) {
        int64_t c = qc[k];
        if (c < 0 || c >= n) return ORC_EINVAL;
        int p = deg[c];
        int m = (int)(coff[c + 1] - coff[c]) - 1;
        curve_eval(p, knots + koff[c], m, cps + 3 * coff[c], w ? w + coff[c] : NULL, t[k], out + 9 * k,
                   out + 9 * k + 3, out + 9 * k + 6);
    }
    return ORC_OK;
}

/* w: NULL (non-rational) or the weights [coff[n]] of every control point */
int orc_eval_surfaces(int64_t n, const int32_t* pu, const int32_t* pv, const int32_t* nu,
                      const int32_t* nv, const int64_t* kuoff, const double* ku,
                      const int64_t* kvoff, const double* kv, const int64_t* coff,
                      const double* cps, const double* w, int64_t nq, const int32_t* qs, const double* uv,
                      double* out /* [nq][6][3] */)
{
    for (int64_t k = 0; k < nq; ++k) {
        int64_t s = qs[k];
        if (s < 0 || s >= n) return ORC_EINVAL;
        surface_eval(pu[s], pv[s], ku + kuoff[s], nu[s] - 1, kv + kvoff[s], nv[s] - 1, cps + 3 * coff[s],
                     w ? w + coff[s] : NULL, nv[s], uv[2 * k], uv[2 * k + 1], out + 18 * k);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* textbook Boehm knot insertion (cross-check of Sec. 4.2.1)            */
/* ------------------------------------------------------------------ */

/* Inserts every interior knot of the valid range until its multiplicity is p
 * (one knot at a time, textbook rule P'_i = a_i P_i + (1 - a_i) P_{i-1}),
 * then reads the Bezier points of each non-empty span.  Q: [cap][p+1][3]. */
int orc_boehm_bezier(int p, const double* U0, int64_t nU0, const double* P0, int64_t nP0,
                     double* Q, int64_t cap, int64_t* nspans)
{
    if (p < 1 || p > OMAXP || nU0 != nP0 + p + 1) return ORC_EINVAL;
    int64_t capU = nU0 * (p + 1) + 8, capP = capU;
    double* U = (double*)malloc(sizeof(double) * (size_t)capU);
    double* P = (double*)malloc(sizeof(double) * 3 * (size_t)capP);
    double* Pn = (double*)malloc(sizeof(double) * 3 * (size_t)capP);
    memcpy(U, U0, sizeof(double) * (size_t)nU0);
    memcpy(P, P0, sizeof(double) * 3 * (size_t)nP0);
    int64_t nU = nU0, nP = nP0;
    double lo = U0[p], hi = U0[nP0]; /* valid range [t_p, t_{m+1}] */
    int64_t i = 0;
    while (i < nU) {
        double x = U[i];
        int64_t mult = 0;
        while (i + mult < nU && U[i + mult] == x) ++mult;
        if (x >= lo && x <= hi) {
            while (mult < p) {
                /* insert x once: k with U[k] <= x < U[k+1] (k = last index of x) */
                int64_t k = i + mult - 1;
                for (int64_t j = 0; j < nP + 1; ++j) {
                    if (j <= k - p) {
                        memcpy(Pn + 3 * j, P + 3 * j, sizeof(double) * 3);
                    } else if (j <= k) {
                        double a = (x - U[j]) / (U[j + p] - U[j]);
                        for (int c = 0; c < 3; ++c)
                            Pn[3 * j + c] = a * P[3 * j + c] + (1.0 - a) * P[3 * (j - 1) + c];
                    } else {
                        memcpy(Pn + 3 * j, P + 3 * (j - 1), sizeof(double) * 3);
                    }
                }
                memcpy(P, Pn, sizeof(double) * 3 * (size_t)(nP + 1));
                ++nP;
                memmove(U + k + 2, U + k + 1, sizeof(double) * (size_t)(nU - k - 1));
                U[k + 1] = x;
                ++nU;
                ++mult;
            }
        }
        i += mult;
    }
    int64_t ns = 0;
    int m = (int)nP - 1;
    for (int q = p; q <= m; ++q) {
        if (!(U[q] < U[q + 1])) continue;
        if (ns < cap)
            memcpy(Q + (size_t)ns * 3 * (p + 1), P + 3 * (q - p), sizeof(double) * 3 * (size_t)(p + 1));
        ++ns;
    }
    *nspans = ns;
    free(U); free(P); free(Pn);
    return ns <= cap ? ORC_OK : ORC_ENOSPACE;
}

/* ------------------------------------------------------------------ */
/* the paper's span-wise matrix route, built in the local parameter u   */
/* (Sec. 4.2.1, Eqs. bsplinematrix, Mqpt, decomfinal)                    */
/* ------------------------------------------------------------------ */

/* Bezier points Q[0..p] of span q.  Step 1: power-basis coefficients in
 * u = (t - t_q)/(t_{q+1} - t_q) of N_{q-p..q,p} by the Cox-de Boor recursion
 * on polynomials (this is the product M_{q,p,T} A_{q,p,T} of the paper, formed
 * directly in u).  Step 2: c = (M A) P.  Step 3: Q = B_p^{-1} c with
 * (B_p^{-1})_{ij} = C(i,j)/C(p,j), j <= i.
 * Pl points at P_{q-p} (p+1 consecutive control points, xyz). */
static void span_bezier(int p, const double* U, int q, const double* Pl, double* Q)
{
    double poly[ONP + 1][ONP + 1], nw[ONP + 1][ONP + 1];
    double du = U[q + 1] - U[q];
    poly[0][0] = 1.0;
    for (int k = 1; k <= p; ++k) {
        for (int j = 0; j <= k; ++j) {
            int i = q - k + j;
            for (int e = 0; e <= k; ++e) nw[j][e] = 0.0;
            if (j >= 1) { /* ((t_q - t_i) + du u)/(t_{i+k} - t_i) * N_{i,k-1} */
                double den = U[i + k] - U[i];
                if (den != 0.0) {
                    double a = (U[q] - U[i]) / den, b = du / den;
                    for (int e = 0; e <= k - 1; ++e) {
                        nw[j][e] = nw[j][e] + a * poly[j - 1][e];
                        nw[j][e + 1] = nw[j][e + 1] + b * poly[j - 1][e];
                    }
                }
            }
            if (j <= k - 1) { /* ((t_{i+k+1} - t_q) - du u)/(t_{i+k+1} - t_{i+1}) * N_{i+1,k-1} */
                double den = U[i + k + 1] - U[i + 1];
                if (den != 0.0) {
                    double a = (U[i + k + 1] - U[q]) / den, b = -du / den;
                    for (int e = 0; e <= k - 1; ++e) {
                        nw[j][e] = nw[j][e] + a * poly[j][e];
                        nw[j][e + 1] = nw[j][e + 1] + b * poly[j][e];
                    }
                }
            }
        }
        for (int j = 0; j <= k; ++j)
            for (int e = 0; e <= k; ++e) poly[j][e] = nw[j][e];
    }
    double cc[ONP + 1][3];
    for (int e = 0; e <= p; ++e)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int j = 0; j <= p; ++j) s = s + poly[j][e] * Pl[3 * j + c];
            cc[e][c] = s;
        }
    for (int i = 0; i <= p; ++i)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int e = 0; e <= i; ++e) s = s + (binom(i, e) / binom(p, e)) * cc[e][c];
            Q[3 * i + c] = s;
        }
}

/* Bezier points Q[0..p] of span q from the blossom (polar form) of the
 * span's polynomial: Q_j = f(t_q, .., t_q, t_{q+1}, .., t_{q+1}) with p - j
 * arguments t_q followed by j arguments t_{q+1}, each by de Boor's algorithm
 * with the arguments in that order: d_i = (1 - a) d_{i-1} + a d_i, a = (x -
 * t_i)/(t_{i+p+1-r} - t_i) for r = 1..p, i = q..q-p+r downwards.  Every a
 * lies in [0, 1] (x is t_q or t_{q+1}, inside [t_i, t_{i+p+1-r}]), so the
 * points are convex combinations of the span's control points at any
 * degree, whereas the matrix route's power-basis coefficients grow like
 * C(p, p/2) and take as many digits with them. */
static void span_blossom(int p, const double* U, int q, const double* Pl, double* Q)
{
    double d[ONP][3];
    for (int j = 0; j <= p; ++j) {
        for (int i = 0; i <= p; ++i)
            for (int c = 0; c < 3; ++c) d[i][c] = Pl[3 * i + c];
        for (int r = 1; r <= p; ++r) {
            double x = r <= p - j ? U[q] : U[q + 1];
            for (int i = p; i >= r; --i) {
                int g = q - p + i;
                double a = (x - U[g]) / (U[g + p + 1 - r] - U[g]);
                for (int c = 0; c < 3; ++c) d[i][c] = (1.0 - a) * d[i - 1][c] + a * d[i][c];
            }
        }
        for (int c = 0; c < 3; ++c) Q[3 * j + c] = d[p][c];
    }
}

/* the extraction the decomposition uses: the matrix route up to degree
 * OMATP, the blossom above it */
static void span_extract(int p, const double* U, int q, const double* Pl, double* Q)
{
    if (p <= OMATP) span_bezier(p, U, q, Pl, Q);
    else span_blossom(p, U, q, Pl, Q);
}

int orc_span_blossom(int p, const double* U, int64_t nU, const double* P, int64_t nP, double* Q, int64_t cap,
                     int64_t* nspans)
{
    if (p < 1 || p > OMAXP || nU != nP + p + 1) return ORC_EINVAL;
    int64_t ns = 0;
    for (int q = p; q <= (int)nP - 1; ++q) {
        if (!(U[q] < U[q + 1])) continue;
        if (ns < cap) span_blossom(p, U, q, P + 3 * (q - p), Q + (size_t)ns * 3 * (p + 1));
        ++ns;
    }
    *nspans = ns;
    return ns <= cap ? ORC_OK : ORC_ENOSPACE;
}

/* all non-empty spans of one curve by the matrix route (exported for pins) */
int orc_span_bezier(int p, const double* U, int64_t nU, const double* P, int64_t nP,
                    double* Q, int64_t cap, int64_t* nspans)
{
    if (p < 1 || p > OMAXP || nU != nP + p + 1) return ORC_EINVAL;
    int64_t ns = 0;
    for (int q = p; q <= (int)nP - 1; ++q) {
        if (!(U[q] < U[q + 1])) continue;
        if (ns < cap) span_bezier(p, U, q, P + 3 * (q - p), Q + (size_t)ns * 3 * (p + 1));
        ++ns;
    }
    *nspans = ns;
    return ns <= cap ? ORC_OK : ORC_ENOSPACE;
}

/* ------------------------------------------------------------------ */
/* elevation, G1 reduction, bound, halving (Sec. 4.2.2)                 */
/* ------------------------------------------------------------------ */

/* degree n -> n+1:  Q'_i = (i/(n+1)) Q_{i-1} + ((n+1-i)/(n+1)) Q_i ; stride s between points
 * of nc coordinates each (3: points, 4: homogeneous points of a rational piece) */
static void elevate_nc(int n, const double* Q, double* E, int s, int nc)
{
    for (int c = 0; c < nc; ++c) {
        E[c] = Q[c];
        E[(n + 1) * s + c] = Q[n * s + c];
    }
    for (int i = 1; i <= n; ++i) {
        double a = (double)i / (double)(n + 1);
        double b = (double)(n + 1 - i) / (double)(n + 1);
        for (int c = 0; c < nc; ++c) E[i * s + c] = a * Q[(i - 1) * s + c] + b * Q[i * s + c];
    }
}

static void elevate(int n, const double* Q, double* E, int s) { elevate_nc(n, Q, E, s, 3); }

/* G1-continuous, L2-optimal reduction of a degree-p Bezier (p > 3) to a cubic.
 * R0 = Q0, R1 = Q0 + (p/3) d0 delta0, R2 = Qp - (p/3) d1 delta1, R3 = Qp
 * (Eq. G1-condition).  delta0, delta1 solve d eps/d delta_i = 0 (Eqs.
 * differentiatedelta0/1), where eps is the L2 error of Eq. epsl.  The 2x2
 * system is derived here from eps directly: substituting R gives
 *   delta0 (A0.d0) + delta1 (A1.d0) = V1.d0
 *   delta0 (B0.d1) + delta1 (B1.d1) = V2.d1
 * with A0 = a g11 d0, A1 = -a g12 d1, B0 = a g21 d0, B1 = -a g22 d1 (g = G_{3,3}),
 * V_r = G^r_{3,p} Q - G^r_{3,3} [Q0,Q0,Qp,Qp].  The printed appendix carries a
 * + in front of the delta1 terms; that sign does not follow from eps and is
 * not used (variant = 1 reproduces the printed sign, for the pin that shows it
 * breaks the optimality condition).  Degenerate systems (zero end tangents,
 * |det| <= 1e-12 |a11 a22|, non-finite or non-positive deltas) fall back to
 * delta0 = delta1 = 1, the C1 end-derivative match. */
static void reduce_g1(int p, const double* Q, int s, double* R, int rs, double* deltas, int variant)
{
    const double* Q0 = Q;
    const double* Q1 = Q + s;
    const double* Qm = Q + (p - 1) * s;
    const double* Qp = Q + p * s;
    double a = (double)p / 3.0;
    double g11 = orc_gram(3, 3, 1, 1), g12 = orc_gram(3, 3, 1, 2);
    double g21 = orc_gram(3, 3, 2, 1), g22 = orc_gram(3, 3, 2, 2);
    double g10 = orc_gram(3, 3, 1, 0), g13 = orc_gram(3, 3, 1, 3);
    double g20 = orc_gram(3, 3, 2, 0), g23 = orc_gram(3, 3, 2, 3);
    double d0[3], d1[3], V1[3], V2[3];
    for (int c = 0; c < 3; ++c) {
        d0[c] = Q1[c] - Q0[c];
        d1[c] = Qp[c] - Qm[c];
        double s1 = 0.0, s2 = 0.0;
        for (int j = 0; j <= p; ++j) {
            s1 = s1 + orc_gram(3, p, 1, j) * Q[j * s + c];
            s2 = s2 + orc_gram(3, p, 2, j) * Q[j * s + c];
        }
        double t1 = ((g10 * Q0[c] + g11 * Q0[c]) + g12 * Qp[c]) + g13 * Qp[c];
        double t2 = ((g20 * Q0[c] + g21 * Q0[c]) + g22 * Qp[c]) + g23 * Qp[c];
        V1[c] = s1 - t1;
        V2[c] = s2 - t2;
    }
    double A0[3], A1[3], B0[3], B1[3];
    for (int c = 0; c < 3; ++c) {
        A0[c] = (a * g11) * d0[c];
        A1[c] = (-a * g12) * d1[c];
        B0[c] = (a * g21) * d0[c];
        B1[c] = (-a * g22) * d1[c];
    }
#define DOT3(x, y) (((x)[0] * (y)[0] + (x)[1] * (y)[1]) + (x)[2] * (y)[2])
    double a11 = DOT3(A0, d0), a12 = DOT3(A1, d0), b1 = DOT3(V1, d0);
    double a21 = DOT3(B0, d1), a22 = DOT3(B1, d1), b2 = DOT3(V2, d1);
#undef DOT3
    if (variant == 1) { /* the appendix's printed sign (not used by the method) */
        a12 = -a12;
        a22 = -a22;
    }
    double det = a11 * a22 - a12 * a21;
    double dl0 = (b1 * a22 - a12 * b2) / det;
    double dl1 = (a11 * b2 - b1 * a21) / det;
    int ok = (det != 0.0) && (fabs(det) > 1e-12 * fabs(a11 * a22)) && isfinite(dl0) &&
             isfinite(dl1) && ((dl0 > 0.0 && dl1 > 0.0) || variant == 1);
    if (!ok) { dl0 = 1.0; dl1 = 1.0; }
    double s0 = a * dl0, s1 = a * dl1;
    for (int c = 0; c < 3; ++c) {
        R[c] = Q0[c];
        R[rs + c] = Q0[c] + s0 * d0[c];
        R[2 * rs + c] = Qp[c] - s1 * d1[c];
        R[3 * rs + c] = Qp[c];
    }
    if (deltas) { deltas[0] = dl0; deltas[1] = dl1; deltas[2] = ok ? 1.0 : 0.0; }
}

/* any degree p >= 1 to a cubic: elevate (p < 3), copy (p = 3), reduce (p > 3) */
static void to_cubic(int p, const double* Q, int s, double* R, int rs)
{
    if (p == 3) {
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) R[i * rs + c] = Q[i * s + c];
    } else if (p > 3) {
        reduce_g1(p, Q, s, R, rs, NULL, 0);
    } else {
        double w[12], x[12];
        for (int i = 0; i <= p; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Q[i * s + c];
        for (int n = p; n < 3; ++n) {
            elevate(n, w, x, 3);
            memcpy(w, x, sizeof(double) * 3 * (size_t)(n + 2));
        }
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) R[i * rs + c] = w[3 * i + c];
    }
}

/* max_i |Q_i - (R elevated to p)_i|^2 : an upper bound of max_u |Q(u)-R(u)|^2
 * because Bernstein weights are a convex partition of unity (p >= 3). */
static double bound2_curve(int p, const double* Q, int s, const double* R, int rs)
{
    double w[(ONP + 1) * 3], x[(ONP + 1) * 3];
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c) w[3 * i + c] = R[i * rs + c];
    for (int n = 3; n < p; ++n) {
        elevate(n, w, x, 3);
        memcpy(w, x, sizeof(double) * 3 * (size_t)(n + 2));
    }
    double b = 0.0;
    for (int i = 0; i <= p; ++i) {
        double dx = Q[i * s + 0] - w[3 * i], dy = Q[i * s + 1] - w[3 * i + 1], dz = Q[i * s + 2] - w[3 * i + 2];
        double e = (dx * dx + dy * dy) + dz * dz;
        if (e > b) b = e;
    }
    return b;
}

/* de Casteljau split at z = 1/2 (the matrix S(1/2) of Eq. subLandR); points
 * of nc coordinates (3, or 4 for homogeneous points) at stride s */
static void halve_nc(int p, const double* Q, int s, int nc, double* L, double* Rr)
{
    double w[ONP + 1][4];
    for (int i = 0; i <= p; ++i)
        for (int c = 0; c < nc; ++c) w[i][c] = Q[i * s + c];
    for (int c = 0; c < nc; ++c) { L[c] = w[0][c]; Rr[p * s + c] = w[p][c]; }
    for (int r = 1; r <= p; ++r) {
        for (int i = 0; i <= p - r; ++i)
            for (int c = 0; c < nc; ++c) w[i][c] = (w[i][c] + w[i + 1][c]) * 0.5;
        for (int c = 0; c < nc; ++c) { L[r * s + c] = w[0][c]; Rr[(p - r) * s + c] = w[p - r][c]; }
    }
}

static void halve(int p, const double* Q, int s, double* L, double* Rr) { halve_nc(p, Q, s, 3, L, Rr); }

/* exported single-step helpers for the pins */
int orc_reduce_g1(int p, const double* Q, double* R, double* deltas, int variant)
{
    if (p <= 3 || p > OMAXP) return ORC_EINVAL;
    reduce_g1(p, Q, 3, R, 3, deltas, variant);
    return ORC_OK;
}
int orc_to_cubic(int p, const double* Q, double* R)
{
    if (p < 1 || p > OMAXP) return ORC_EINVAL;
    to_cubic(p, Q, 3, R, 3);
    return ORC_OK;
}
double orc_bound2(int p, const double* Q, const double* R) { return bound2_curve(p, Q, 3, R, 3); }
int orc_halve(int p, const double* Q, double* L, double* R)
{
    if (p < 1 || p > OMAXP) return ORC_EINVAL;
    halve(p, Q, 3, L, R);
    return ORC_OK;
}
int orc_elevate(int n, const double* Q, double* E)
{
    if (n < 1 || n >= OMAXP) return ORC_EINVAL;
    elevate(n, Q, E, 3);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* error-controlled curve decomposition (Sec. 4.2.2)                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int p;
    double thr2;
    double tq, tq1;
    int64_t count, cap, span_first;
    double* ctrl;   /* [cap][4][3] */
    double* prange; /* [cap][2] */
    int maxdepth;
    int notconv;
} curve_ctx;

/* parameter of the dyadic point k/2^L of span [tq, tq1] */
static double dyadic_t(double tq, double tq1, int64_t k, int L)
{
    if (k == 0) return tq;
    if (k == ((int64_t)1 << L)) return tq1;
    return tq + (tq1 - tq) * ldexp((double)k, -L);
}

/* accept the cubic of this node or split it at the midpoint of its parameter
 * interval; children are re-reduced from the ORIGINAL degree-p piece, so their
 * shared end point lies on the original curve (Sec. 4.2.2, control-polygon
 * modification, midpoint reading) */
static void curve_node(curve_ctx* X, const double* Q, int L, int64_t k)
{
    double R[12];
    int p = X->p;
    to_cubic(p, Q, 3, R, 3);
    int accept = 1;
    if (p > 3) accept = bound2_curve(p, Q, 3, R, 3) <= X->thr2;
    if (!accept && (L >= ODEPTH || X->count - X->span_first >= OLEAFCAP)) { accept = 1; X->notconv = 1; }
    if (accept) {
        if (X->count < X->cap && X->ctrl) {
            memcpy(X->ctrl + 12 * X->count, R, sizeof(R));
            X->prange[2 * X->count] = dyadic_t(X->tq, X->tq1, k, L);
            X->prange[2 * X->count + 1] = dyadic_t(X->tq, X->tq1, k + 1, L);
        }
        X->count++;
        if (L > X->maxdepth) X->maxdepth = L;
        return;
    }
    double Lq[(ONP + 1) * 3], Rq[(ONP + 1) * 3];
    halve(p, Q, 3, Lq, Rq);
    curve_node(X, Lq, L + 1, 2 * k);
    curve_node(X, Rq, L + 1, 2 * k + 1);
}

/* diagonal of the axis-aligned box of np points */
static double box_diag(const double* P, int64_t np)
{
    double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int64_t i = 0; i < np; ++i)
        for (int c = 0; c < 3; ++c) {
            if (P[3 * i + c] < lo[c]) lo[c] = P[3 * i + c];
            if (P[3 * i + c] > hi[c]) hi[c] = P[3 * i + c];
        }
    double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return sqrt((dx * dx + dy * dy) + dz * dz);
}

static int check_knots(int p, const double* U, int64_t nU, int64_t nP)
{
    if (p < 1 || p > OMAXP || nP < p + 1 || nU != nP + p + 1) return 0;
    for (int64_t i = 0; i < nU; ++i) {
        if (!isfinite(U[i])) return 0;
        if (i > 0 && U[i] < U[i - 1]) return 0;
    }
    return U[p] < U[nP];
}

/* ------------------------------------------------------------------ */
/* rational curves (NURBS): homogeneous decomposition                    */
/* ------------------------------------------------------------------ */
/* A rational curve is C = A/W with A = sum N_i w_i P_i, W = sum N_i w_i,
 * both non-rational B-splines of the homogeneous control points (w_i P_i,
 * w_i).  The span-wise matrix route is linear in the control points, so it
 * gives the span's rational Bezier piece as homogeneous points H_j = (W_j Q_j,
 * W_j), and the midpoint halving of Eq. subLandR applies to H unchanged.  The
 * paper's pieces are polynomial (its method covers non-rational splines
 * only); a rational piece is replaced by the C1 Hermite cubic R of its end
 * points and end derivatives, bounded and subdivided as below, so that the
 * query tables hold cubic Beziers whatever the input. */

/* homogeneous Bezier points H [p+1][4] of span q (the matrix route applied
 * to (w_i P_i) and to (w_i), which are products of one rounding each) */
static void rspan_bezier(int p, const double* U, int q, const double* Pl, const double* wl, double* H)
{
    double hp[(ONP + 1) * 3], hw[(ONP + 1) * 3], Qp[(ONP + 1) * 3], Qw[(ONP + 1) * 3];
    for (int j = 0; j <= p; ++j) {
        for (int c = 0; c < 3; ++c) hp[3 * j + c] = wl[j] * Pl[3 * j + c];
        hw[3 * j] = wl[j];
        hw[3 * j + 1] = 0.0;
        hw[3 * j + 2] = 0.0;
    }
    span_extract(p, U, q, hp, Qp);
    span_extract(p, U, q, hw, Qw);
    for (int j = 0; j <= p; ++j) {
        for (int c = 0; c < 3; ++c) H[4 * j + c] = Qp[3 * j + c];
        H[4 * j + 3] = Qw[3 * j];
    }
}

/* the C1 Hermite cubic R [4][3] of the rational piece H: R_0 = C(0), R_3 =
 * C(1), R_1 = C(0) + C'(0)/3, R_2 = C(1) - C'(1)/3, with the end derivatives
 * of a rational Bezier (quotient rule at u = 0 and 1)
 *   C'(0) = p (H_1 - W_1 C(0)) / W_0,   C'(1) = p (W_{p-1} C(1) - H_{p-1}) / W_p
 * (the numerator parts of H_1 and H_{p-1} written H_1, H_{p-1}). */
static void rhermite(int p, const double* H, double* R)
{
    const double a = (double)p / 3.0;
    const double* h0 = H;
    const double* h1 = H + 4;
    const double* hm = H + 4 * (p - 1);
    const double* hp = H + 4 * p;
    for (int c = 0; c < 3; ++c) {
        double c0 = h0[c] / h0[3], c1 = hp[c] / hp[3];
        R[c] = c0;
        R[3 + c] = c0 + a * ((h1[c] - h1[3] * c0) / h0[3]);
        R[6 + c] = c1 + a * ((hm[c] - hm[3] * c1) / hp[3]);
        R[9 + c] = c1;
    }
}

/* certified bound of max_u |C(u) - R(u)|^2 on [0, 1]:
 *   C - R = (A - W R) / W,
 * A - W R is a polynomial of degree p + 3 whose Bernstein coefficients are
 * those of A elevated three times minus those of the product W R,
 *   (W R)_k = sum_j [C(p, j) C(3, k - j) / C(p + 3, k)] W_j R_{k-j};
 * Bernstein weights are a convex partition of unity, so the largest
 * coefficient norm bounds |A - W R|, and W >= min_j W_j > 0. */
static double rbound2(int p, const double* H, const double* R)
{
    double e[(ONP + 4) * 4], x[(ONP + 4) * 4];
    for (int i = 0; i < 4 * (p + 1); ++i) e[i] = H[i];
    for (int n = p; n < p + 3; ++n) {
        elevate_nc(n, e, x, 4, 4);
        memcpy(e, x, sizeof(double) * 4 * (size_t)(n + 2));
    }
    double wmin = H[3];
    for (int j = 1; j <= p; ++j)
        if (H[4 * j + 3] < wmin) wmin = H[4 * j + 3];
    double b = 0.0;
    for (int k = 0; k <= p + 3; ++k) {
        double s[3] = { 0.0, 0.0, 0.0 };
        int jlo = k - 3 > 0 ? k - 3 : 0, jhi = k < p ? k : p;
        for (int j = jlo; j <= jhi; ++j) {
            double cf = (binom(p, j) * binom(3, k - j)) / binom(p + 3, k);
            for (int c = 0; c < 3; ++c) s[c] = s[c] + (cf * H[4 * j + 3]) * R[3 * (k - j) + c];
        }
        double dx = e[4 * k] - s[0], dy = e[4 * k + 1] - s[1], dz = e[4 * k + 2] - s[2];
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 > b) b = d2;
    }
    return b / (wmin * wmin);
}

/* the rational counterpart of curve_node: the Hermite cubic of the node is
 * accepted when its bound meets the tolerance, else the homogeneous piece is
 * split at its parameter midpoint (same caps) */
static void rcurve_node(curve_ctx* X, const double* H, int L, int64_t k)
{
    double R[12];
    int p = X->p;
    rhermite(p, H, R);
    int accept = rbound2(p, H, R) <= X->thr2;
    if (!accept && (L >= ODEPTH || X->count - X->span_first >= OLEAFCAP)) { accept = 1; X->notconv = 1; }
    if (accept) {
        if (X->count < X->cap && X->ctrl) {
            memcpy(X->ctrl + 12 * X->count, R, sizeof(R));
            X->prange[2 * X->count] = dyadic_t(X->tq, X->tq1, k, L);
            X->prange[2 * X->count + 1] = dyadic_t(X->tq, X->tq1, k + 1, L);
        }
        X->count++;
        if (L > X->maxdepth) X->maxdepth = L;
        return;
    }
    double Lh[(ONP + 1) * 4], Rh[(ONP + 1) * 4];
    halve_nc(p, H, 4, 4, Lh, Rh);
    rcurve_node(X, Lh, L + 1, 2 * k);
    rcurve_node(X, Rh, L + 1, 2 * k + 1);
}

/* weights of a curve: 1 = rational (not all equal), 0 = all equal (the
 * curve is then the non-rational one: A/W = sum N_i P_i, the basis being a
 * partition of unity), -1 = a weight that is not finite and positive */
static int weights_kind(const double* w, int64_t nP)
{
    int rat = 0;
    for (int64_t i = 0; i < nP; ++i) {
        if (!(isfinite(w[i]) && w[i] > 0.0)) return -1;
        if (w[i] != w[0]) rat = 1;
    }
    return rat;
}

/* exported for the pins */
int orc_rspan_bezier(int p, const double* U, int64_t nU, const double* P, const double* w, int64_t nP,
                     double* H, int64_t cap, int64_t* nspans)
{
    if (p < 1 || p > OMAXP || nU != nP + p + 1) return ORC_EINVAL;
    int64_t ns = 0;
    for (int q = p; q <= (int)nP - 1; ++q) {
        if (!(U[q] < U[q + 1])) continue;
        if (ns < cap) rspan_bezier(p, U, q, P + 3 * (q - p), w + (q - p), H + (size_t)ns * 4 * (p + 1));
        ++ns;
    }
    *nspans = ns;
    return ns <= cap ? ORC_OK : ORC_ENOSPACE;
}
int orc_rhermite(int p, const double* H, double* R)
{
    if (p < 1 || p > OMAXP) return ORC_EINVAL;
    rhermite(p, H, R);
    return ORC_OK;
}
double orc_rbound2(int p, const double* H, const double* R) { return rbound2(p, H, R); }
int orc_rhalve(int p, const double* H, double* L, double* R)
{
    if (p < 1 || p > OMAXP) return ORC_EINVAL;
    halve_nc(p, H, 4, 4, L, R);
    return ORC_OK;
}

/* decomposes curve c with its segments written from index `first` (when the
 * arrays are given and fit); returns the count, or -1 for invalid data.
 * w: NULL, or the weights of every control point of the set (a curve whose
 * weights are all equal takes the non-rational route) */
static int64_t decompose_one_curve(int64_t c, const int32_t* deg, const int64_t* koff, const double* knots,
                                   const int64_t* coff, const double* cps, const double* w, double tol_rel,
                                   int64_t first, int64_t cap, double* ctrl, double* prange, int* maxdepth,
                                   int* notconv)
{
    int p = deg[c];
    int64_t nP = coff[c + 1] - coff[c], nU = koff[c + 1] - koff[c];
    const double* U = knots + koff[c];
    const double* P = cps + 3 * coff[c];
    const double* wc = w ? w + coff[c] : NULL;
    if (!check_knots(p, U, nU, nP)) return -1;
    for (int64_t i = 0; i < 3 * nP; ++i) if (!isfinite(P[i])) return -1;
    int rat = wc ? weights_kind(wc, nP) : 0;
    if (rat < 0) return -1;
    double thr = tol_rel * box_diag(P, nP);
    curve_ctx X;
    X.p = p; X.thr2 = thr * thr; X.cap = cap; X.maxdepth = 0; X.notconv = 0;
    X.ctrl = ctrl; X.prange = prange;
    X.count = first;
    for (int q = p; q <= (int)nP - 1; ++q) {
        if (!(U[q] < U[q + 1])) continue;
        X.tq = U[q]; X.tq1 = U[q + 1];
        X.span_first = X.count;
        if (rat) {
            double H[(ONP + 1) * 4];
            rspan_bezier(p, U, q, P + 3 * (q - p), wc + (q - p), H);
            rcurve_node(&X, H, 0, 0);
        } else {
            double Q[(ONP + 1) * 3];
            span_extract(p, U, q, P + 3 * (q - p), Q);
            curve_node(&X, Q, 0, 0);
        }
    }
    *maxdepth = X.maxdepth;
    *notconv = X.notconv;
    return X.count - first;
}

/* seg_off[n+1] always written; ctrl/prange written when cap suffices.
 * returns ORC_ENOSPACE when the total exceeds cap (counts still valid).
 * Curves are independent: counted in parallel, offsets by a prefix sum, then
 * filled in parallel. */
int orc_decompose_curves(int64_t n, const int32_t* deg, const int64_t* koff, const double* knots,
                         const int64_t* coff, const double* cps, const double* w, double tol_rel, int64_t* seg_off,
                         int64_t cap, double* ctrl, double* prange, int64_t* total, int* maxdepth)
{
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int md = 0, nc = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(max : md) reduction(| : nc, bad)
    for (int64_t c = 0; c < n; ++c) {
        int m1 = 0, n1 = 0;
        cnt[c] = decompose_one_curve(c, deg, koff, knots, coff, cps, w, tol_rel, 0, 0, NULL, NULL, &m1, &n1);
        if (cnt[c] < 0) bad = 1;
        if (m1 > md) md = m1;
        nc |= n1;
    }
    if (bad) { free(cnt); return ORC_EINVAL; }
    seg_off[0] = 0;
    for (int64_t c = 0; c < n; ++c) seg_off[c + 1] = seg_off[c] + cnt[c];
    int64_t tot = seg_off[n];
    if (ctrl && tot <= cap) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t c = 0; c < n; ++c) {
            int m1, n1;
            decompose_one_curve(c, deg, koff, knots, coff, cps, w, tol_rel, seg_off[c], cap, ctrl, prange, &m1,
                                &n1);
        }
    }
    free(cnt);
    *total = tot;
    if (maxdepth) *maxdepth = md;
    if (nc) return ORC_ENOTCONV;
    return tot <= cap ? ORC_OK : ORC_ENOSPACE;
}

/* ------------------------------------------------------------------ */
/* error-controlled surface decomposition (tensor-product reading)       */
/* ------------------------------------------------------------------ */

#define SMAXP 15 /* surfaces: degree <= 15 per direction in the oracle */
#define SNP (SMAXP + 1)

typedef struct {
    int pu, pv;
    double thr2;
    double u0, u1, v0, v1; /* span pair parameter box */
    int64_t count, cap, span_first;
    double* ctrl;   /* [cap][4][4][3] */
    double* prange; /* [cap][4] */
    int maxdepth, notconv;
} surf_ctx;

/* a net of (pu+1) x (pv+1) points (index a along u), stored flat with a fixed
 * row length: point (a, b) at NETI(a, b) */
#define NETI(a, b) (((a) * SNP + (b)) * 3)
#define NETN (SNP * SNP * 3)

/* reduce along u for every v column, then along v for every u row */
static void surf_to_bicubic(int pu, int pv, const double* Q, double* R /* [4][4][3] flat */)
{
    double Rp[4 * SNP * 3];
    for (int j = 0; j <= pv; ++j) {
        double col[SNP * 3], r[12];
        for (int i = 0; i <= pu; ++i)
            for (int c = 0; c < 3; ++c) col[3 * i + c] = Q[NETI(i, j) + c];
        to_cubic(pu, col, 3, r, 3);
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) Rp[NETI(i, j) + c] = r[3 * i + c];
    }
    for (int i = 0; i < 4; ++i) {
        double r[12];
        to_cubic(pv, Rp + NETI(i, 0), 3, r, 3);
        for (int j = 0; j < 4; ++j)
            for (int c = 0; c < 3; ++c) R[(i * 4 + j) * 3 + c] = r[3 * j + c];
    }
}

static void elevate_to(int from, int to, double* w /* [SNP*3] */)
{
    double x[SNP * 3];
    for (int n = from; n < to; ++n) {
        elevate(n, w, x, 3);
        memcpy(w, x, sizeof(double) * 3 * (size_t)(n + 2));
    }
}

/* certified bound at degrees (eu, ev) = (max(pu,3), max(pv,3)):
 * Q elevated along u then v where its degree is below 3; R elevated along v
 * then u where the original degree is above 3. */
static double surf_bound2(int pu, int pv, const double* Q, const double* R)
{
    int eu = pu > 3 ? pu : 3, ev = pv > 3 ? pv : 3;
    double* Qe = (double*)malloc(sizeof(double) * NETN);
    double* Re = (double*)malloc(sizeof(double) * NETN);
    for (int j = 0; j <= pv; ++j) {
        double w[SNP * 3];
        for (int i = 0; i <= pu; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Q[NETI(i, j) + c];
        elevate_to(pu, eu, w);
        for (int i = 0; i <= eu; ++i)
            for (int c = 0; c < 3; ++c) Qe[NETI(i, j) + c] = w[3 * i + c];
    }
    for (int i = 0; i <= eu; ++i) {
        double w[SNP * 3];
        for (int j = 0; j <= pv; ++j)
            for (int c = 0; c < 3; ++c) w[3 * j + c] = Qe[NETI(i, j) + c];
        elevate_to(pv, ev, w);
        for (int j = 0; j <= ev; ++j)
            for (int c = 0; c < 3; ++c) Qe[NETI(i, j) + c] = w[3 * j + c];
    }
    for (int i = 0; i < 4; ++i) {
        double w[SNP * 3];
        for (int j = 0; j < 4; ++j)
            for (int c = 0; c < 3; ++c) w[3 * j + c] = R[(i * 4 + j) * 3 + c];
        elevate_to(3, ev, w);
        for (int j = 0; j <= ev; ++j)
            for (int c = 0; c < 3; ++c) Re[NETI(i, j) + c] = w[3 * j + c];
    }
    for (int j = 0; j <= ev; ++j) {
        double w[SNP * 3];
        for (int i = 0; i < 4; ++i)
            for (int c = 0; c < 3; ++c) w[3 * i + c] = Re[NETI(i, j) + c];
        elevate_to(3, eu, w);
        for (int i = 0; i <= eu; ++i)
            for (int c = 0; c < 3; ++c) Re[NETI(i, j) + c] = w[3 * i + c];
    }
    double b = 0.0;
    for (int i = 0; i <= eu; ++i)
        for (int j = 0; j <= ev; ++j) {
            const double* a = Qe + NETI(i, j);
            const double* r = Re + NETI(i, j);
            double dx = a[0] - r[0], dy = a[1] - r[1], dz = a[2] - r[2];
            double e = (dx * dx + dy * dy) + dz * dz;
            if (e > b) b = e;
        }
    free(Qe); free(Re);
    return b;
}

/* squared certified deviation of the reduction along one direction alone:
 * every column (dir 0, along u) or row (dir 1, along v) of the net reduced
 * to a cubic and bounded against itself (degree > 3 in that direction) */
static double surf_dir_dev2(int pu, int pv, const double* Q, int dir)
{
    double b = 0.0;
    if (dir == 0) {
        for (int j = 0; j <= pv; ++j) {
            double col[SNP * 3], r[12];
            for (int i = 0; i <= pu; ++i)
                for (int c = 0; c < 3; ++c) col[3 * i + c] = Q[NETI(i, j) + c];
            to_cubic(pu, col, 3, r, 3);
            double e = bound2_curve(pu, col, 3, r, 3);
            if (e > b) b = e;
        }
    } else {
        for (int i = 0; i <= pu; ++i) {
            double row[SNP * 3], r[12];
            for (int j = 0; j <= pv; ++j)
                for (int c = 0; c < 3; ++c) row[3 * j + c] = Q[NETI(i, j) + c];
            to_cubic(pv, row, 3, r, 3);
            double e = bound2_curve(pv, row, 3, r, 3);
            if (e > b) b = e;
        }
    }
    return b;
}

/* split direction: the reduced direction if only one is reduced, else the
 * one whose reduction alone deviates more (ties -> u) */
static int surf_split_dir(int pu, int pv, const double* Q)
{
    if (pu > 3 && pv <= 3) return 0;
    if (pv > 3 && pu <= 3) return 1;
    return surf_dir_dev2(pu, pv, Q, 0) >= surf_dir_dev2(pu, pv, Q, 1) ? 0 : 1;
}

static void surf_node(surf_ctx* X, const double* Q, int Lu, int64_t ku, int Lv, int64_t kv)
{
    int pu = X->pu, pv = X->pv;
    double R[48];
    surf_to_bicubic(pu, pv, Q, R);
    int accept = 1;
    if (pu > 3 || pv > 3) accept = surf_bound2(pu, pv, Q, R) <= X->thr2;
    if (!accept && (Lu + Lv >= ODEPTH || X->count - X->span_first >= OLEAFCAP)) { accept = 1; X->notconv = 1; }
    if (accept) {
        if (X->count < X->cap && X->ctrl) {
            memcpy(X->ctrl + 48 * X->count, R, sizeof(R));
            double* pr = X->prange + 4 * X->count;
            pr[0] = dyadic_t(X->u0, X->u1, ku, Lu);
            pr[1] = dyadic_t(X->u0, X->u1, ku + 1, Lu);
            pr[2] = dyadic_t(X->v0, X->v1, kv, Lv);
            pr[3] = dyadic_t(X->v0, X->v1, kv + 1, Lv);
        }
        X->count++;
        if (Lu + Lv > X->maxdepth) X->maxdepth = Lu + Lv;
        return;
    }
    int dir = surf_split_dir(pu, pv, Q);
    double* A = (double*)malloc(sizeof(double) * NETN);
    double* B = (double*)malloc(sizeof(double) * NETN);
    if (dir == 0) {
        for (int j = 0; j <= pv; ++j) {
            double col[SNP * 3], l[SNP * 3], r[SNP * 3];
            for (int i = 0; i <= pu; ++i)
                for (int c = 0; c < 3; ++c) col[3 * i + c] = Q[NETI(i, j) + c];
            halve(pu, col, 3, l, r);
            for (int i = 0; i <= pu; ++i)
                for (int c = 0; c < 3; ++c) { A[NETI(i, j) + c] = l[3 * i + c]; B[NETI(i, j) + c] = r[3 * i + c]; }
        }
        surf_node(X, A, Lu + 1, 2 * ku, Lv, kv);
        surf_node(X, B, Lu + 1, 2 * ku + 1, Lv, kv);
    } else {
        for (int i = 0; i <= pu; ++i) {
            double l[SNP * 3], r[SNP * 3];
            halve(pv, Q + NETI(i, 0), 3, l, r);
            for (int j = 0; j <= pv; ++j)
                for (int c = 0; c < 3; ++c) { A[NETI(i, j) + c] = l[3 * j + c]; B[NETI(i, j) + c] = r[3 * j + c]; }
        }
        surf_node(X, A, Lu, ku, Lv + 1, 2 * kv);
        surf_node(X, B, Lu, ku, Lv + 1, 2 * kv + 1);
    }
    free(A); free(B);
}

/* Bezier net of span pair (qu, qv): the curve matrix route along u for every
 * v index of the local window, then along v for every u row. */
static void surf_span_bezier(int pu, int pv, const double* U, int qu, const double* V, int qv,
                             const double* P, int nv, double* Q)
{
    double* T1 = (double*)malloc(sizeof(double) * NETN);
    for (int b = 0; b <= pv; ++b) {
        double loc[SNP * 3], out[SNP * 3];
        for (int a = 0; a <= pu; ++a)
            for (int c = 0; c < 3; ++c)
                loc[3 * a + c] = P[3 * ((int64_t)(qu - pu + a) * nv + (qv - pv + b)) + c];
        span_bezier(pu, U, qu, loc, out);
        for (int a = 0; a <= pu; ++a)
            for (int c = 0; c < 3; ++c) T1[NETI(a, b) + c] = out[3 * a + c];
    }
    for (int a = 0; a <= pu; ++a) {
        double out[SNP * 3];
        span_bezier(pv, V, qv, T1 + NETI(a, 0), out);
        for (int b = 0; b <= pv; ++b)
            for (int c = 0; c < 3; ++c) Q[NETI(a, b) + c] = out[3 * b + c];
    }
    free(T1);
}

/* ------------------------------------------------------------------ */
/* rational surfaces: homogeneous decomposition                          */
/* ------------------------------------------------------------------ */
/* The curves' reading carried to tensor-product surfaces: the span pair's
 * piece is the rational tensor Bezier of the homogeneous net H_ab = (W_ab
 * Q_ab, W_ab) that the matrix route gives for (w P, w); a node is replaced
 * by its bicubic Hermite patch (corner values, first partials and twists of
 * the rational piece), accepted when the certified bound of Eq. below meets
 * the tolerance, else halved along the direction whose lines deviate more
 * from their Hermite cubics. */

#define HNETI(a, b) (((a) * SNP + (b)) * 4)
#define HNETN (SNP * SNP * 4)
#define ENP (SNP + 3)                        /* points per direction after elevation by 3 */
#define ENETI(a, b) (((a) * ENP + (b)) * 4)

/* homogeneous net H of span pair (qu, qv): the matrix route applied to the
 * numerator points wP [nu][nv][3] and to (w, 0, 0) */
static void rsurf_span_bezier(int pu, int pv, const double* U, int qu, const double* V, int qv, const double* wP,
                              const double* w3, int nv, double* H)
{
    double* A = (double*)malloc(sizeof(double) * NETN);
    double* B = (double*)malloc(sizeof(double) * NETN);
    surf_span_bezier(pu, pv, U, qu, V, qv, wP, nv, A);
    surf_span_bezier(pu, pv, U, qu, V, qv, w3, nv, B);
    for (int a = 0; a <= pu; ++a)
        for (int b = 0; b <= pv; ++b) {
            for (int c = 0; c < 3; ++c) H[HNETI(a, b) + c] = A[NETI(a, b) + c];
            H[HNETI(a, b) + 3] = B[NETI(a, b)];
        }
    free(A); free(B);
}

/* value, u- and v-partials and twist of the rational piece at corner (ca,
 * cb) in {0,1}^2 of its [0,1]^2 parameters: from A, W and their partials at
 * the corner (differences of the homogeneous net, times the degrees) by
 * the quotient rule */
static void rsurf_corner(int pu, int pv, const double* H, int ca, int cb, double* S, double* Su, double* Sv,
                         double* Suv)
{
    int a0 = ca ? pu : 0, a1 = ca ? pu - 1 : 1, b0 = cb ? pv : 0, b1 = cb ? pv - 1 : 1;
    double su = ca ? -1.0 : 1.0, sv = cb ? -1.0 : 1.0; /* d/du = pu (H_a1 - H_a0) at u = 0, pu (H_a0 - H_a1) at 1 */
    double A[4], Au[4], Av[4], Auv[4];
    for (int c = 0; c < 4; ++c) {
        double h00 = H[HNETI(a0, b0) + c], h10 = H[HNETI(a1, b0) + c];
        double h01 = H[HNETI(a0, b1) + c], h11 = H[HNETI(a1, b1) + c];
        A[c] = h00;
        Au[c] = su * pu * (h10 - h00);
        Av[c] = sv * pv * (h01 - h00);
        Auv[c] = su * sv * (double)pu * (double)pv * (((h11 - h10) - h01) + h00);
    }
    for (int c = 0; c < 3; ++c) {
        S[c] = A[c] / A[3];
        Su[c] = (Au[c] - Au[3] * S[c]) / A[3];
        Sv[c] = (Av[c] - Av[3] * S[c]) / A[3];
        Suv[c] = (((Auv[c] - Au[3] * Sv[c]) - Av[3] * Su[c]) - Auv[3] * S[c]) / A[3];
    }
}

/* the bicubic Hermite patch R [4][4][3] (index i along u): corner values,
 * first partials over 3 and twists over 9 placed in the Bezier net (the
 * corner's point, its neighbours along u and v, and the inner point) */
static void rsurf_hermite(int pu, int pv, const double* H, double* R)
{
    for (int ca = 0; ca < 2; ++ca)
        for (int cb = 0; cb < 2; ++cb) {
            double S[3], Su[3], Sv[3], Suv[3];
            rsurf_corner(pu, pv, H, ca, cb, S, Su, Sv, Suv);
            double su = ca ? -1.0 : 1.0, sv = cb ? -1.0 : 1.0;
            int i0 = ca ? 3 : 0, i1 = ca ? 2 : 1, j0 = cb ? 3 : 0, j1 = cb ? 2 : 1;
            for (int c = 0; c < 3; ++c) {
                R[(i0 * 4 + j0) * 3 + c] = S[c];
                R[(i1 * 4 + j0) * 3 + c] = S[c] + su * (Su[c] / 3.0);
                R[(i0 * 4 + j1) * 3 + c] = S[c] + sv * (Sv[c] / 3.0);
                R[(i1 * 4 + j1) * 3 + c] = ((S[c] + su * (Su[c] / 3.0)) + sv * (Sv[c] / 3.0)) + su * sv * (Suv[c] / 9.0);
            }
        }
}

/* elevate the line of n+1 homogeneous points at stride s by three degrees
 * (into the same line, which must have room for n+4 points) */
static void elevate3_line(int n, double* L, int s)
{
    double a[(ENP + 1) * 4], b[(ENP + 1) * 4];
    for (int i = 0; i <= n; ++i)
        for (int c = 0; c < 4; ++c) a[4 * i + c] = L[i * s + c];
    for (int k = n; k < n + 3; ++k) {
        elevate_nc(k, a, b, 4, 4);
        memcpy(a, b, sizeof(double) * 4 * (size_t)(k + 2));
    }
    for (int i = 0; i <= n + 3; ++i)
        for (int c = 0; c < 4; ++c) L[i * s + c] = a[4 * i + c];
}

/* certified bound of max |S - R|^2 over the piece: S - R = (A - W R)/W with
 * A - W R of degrees (pu + 3, pv + 3); its Bernstein coefficients are A's
 * elevated three times in each direction minus the product
 *   (W R)_kl = sum_ij [C(pu,i) C(3,k-i) / C(pu+3,k)] [C(pv,j) C(3,l-j) / C(pv+3,l)] W_ij R_{k-i,l-j};
 * the largest coefficient norm bounds |A - W R| and W >= min W_ij > 0. */
static double rsurf_bound2(int pu, int pv, const double* H, const double* R)
{
    double* E = (double*)calloc((size_t)ENP * ENP * 4, sizeof(double));
    double wmin = INFINITY;
    for (int a = 0; a <= pu; ++a)
        for (int b = 0; b <= pv; ++b) {
            for (int c = 0; c < 4; ++c) E[ENETI(a, b) + c] = H[HNETI(a, b) + c];
            if (H[HNETI(a, b) + 3] < wmin) wmin = H[HNETI(a, b) + 3];
        }
    for (int b = 0; b <= pv; ++b) elevate3_line(pu, E + ENETI(0, b), ENP * 4);
    for (int a = 0; a <= pu + 3; ++a) elevate3_line(pv, E + ENETI(a, 0), 4);
    double bmax = 0.0;
    for (int k = 0; k <= pu + 3; ++k)
        for (int l = 0; l <= pv + 3; ++l) {
            double sm[3] = { 0.0, 0.0, 0.0 };
            for (int i = (k - 3 > 0 ? k - 3 : 0); i <= (k < pu ? k : pu); ++i) {
                double cu = (binom(pu, i) * binom(3, k - i)) / binom(pu + 3, k);
                for (int j = (l - 3 > 0 ? l - 3 : 0); j <= (l < pv ? l : pv); ++j) {
                    double cv = (binom(pv, j) * binom(3, l - j)) / binom(pv + 3, l);
                    double cw = (cu * cv) * H[HNETI(i, j) + 3];
                    const double* r = R + ((k - i) * 4 + (l - j)) * 3;
                    for (int c = 0; c < 3; ++c) sm[c] = sm[c] + cw * r[c];
                }
            }
            double dx = E[ENETI(k, l)] - sm[0], dy = E[ENETI(k, l) + 1] - sm[1], dz = E[ENETI(k, l) + 2] - sm[2];
            double d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 > bmax) bmax = d2;
        }
    free(E);
    return bmax / (wmin * wmin);
}

/* split direction: the one whose lines (the rational curves of the net along
 * it) deviate more from their Hermite cubics, by the curves' bound (ties:
 * u) */
static int rsurf_split_dir(int pu, int pv, const double* H)
{
    double du = 0.0, dv = 0.0;
    double line[(SNP + 1) * 4], R[12];
    for (int b = 0; b <= pv; ++b) {
        for (int a = 0; a <= pu; ++a)
            for (int c = 0; c < 4; ++c) line[4 * a + c] = H[HNETI(a, b) + c];
        rhermite(pu, line, R);
        double e = rbound2(pu, line, R);
        if (e > du) du = e;
    }
    for (int a = 0; a <= pu; ++a) {
        for (int b = 0; b <= pv; ++b)
            for (int c = 0; c < 4; ++c) line[4 * b + c] = H[HNETI(a, b) + c];
        rhermite(pv, line, R);
        double e = rbound2(pv, line, R);
        if (e > dv) dv = e;
    }
    return du >= dv ? 0 : 1;
}

static void rsurf_node(surf_ctx* X, const double* H, int Lu, int64_t ku, int Lv, int64_t kv)
{
    int pu = X->pu, pv = X->pv;
    double R[48];
    rsurf_hermite(pu, pv, H, R);
    int accept = rsurf_bound2(pu, pv, H, R) <= X->thr2;
    if (!accept && (Lu + Lv >= ODEPTH || X->count - X->span_first >= OLEAFCAP)) { accept = 1; X->notconv = 1; }
    if (accept) {
        if (X->count < X->cap && X->ctrl) {
            memcpy(X->ctrl + 48 * X->count, R, sizeof(R));
            double* pr = X->prange + 4 * X->count;
            pr[0] = dyadic_t(X->u0, X->u1, ku, Lu);
            pr[1] = dyadic_t(X->u0, X->u1, ku + 1, Lu);
            pr[2] = dyadic_t(X->v0, X->v1, kv, Lv);
            pr[3] = dyadic_t(X->v0, X->v1, kv + 1, Lv);
        }
        X->count++;
        if (Lu + Lv > X->maxdepth) X->maxdepth = Lu + Lv;
        return;
    }
    int dir = rsurf_split_dir(pu, pv, H);
    double* A = (double*)malloc(sizeof(double) * HNETN);
    double* B = (double*)malloc(sizeof(double) * HNETN);
    if (dir == 0) {
        for (int j = 0; j <= pv; ++j) halve_nc(pu, H + HNETI(0, j), SNP * 4, 4, A + HNETI(0, j), B + HNETI(0, j));
        rsurf_node(X, A, Lu + 1, 2 * ku, Lv, kv);
        rsurf_node(X, B, Lu + 1, 2 * ku + 1, Lv, kv);
    } else {
        for (int i = 0; i <= pu; ++i) halve_nc(pv, H + HNETI(i, 0), 4, 4, A + HNETI(i, 0), B + HNETI(i, 0));
        rsurf_node(X, A, Lu, ku, Lv + 1, 2 * kv);
        rsurf_node(X, B, Lu, ku, Lv + 1, 2 * kv + 1);
    }
    free(A); free(B);
}

/* exported for the pins; H compact [pu+1][pv+1][4] */
static void compact_to_hnet(int pu, int pv, const double* Hc, double* H)
{
    for (int a = 0; a <= pu; ++a)
        for (int b = 0; b <= pv; ++b)
            for (int c = 0; c < 4; ++c) H[HNETI(a, b) + c] = Hc[((a * (pv + 1)) + b) * 4 + c];
}
int orc_rsurf_hermite(int pu, int pv, const double* Hc, double* R)
{
    if (pu < 1 || pv < 1 || pu > SMAXP || pv > SMAXP) return ORC_EINVAL;
    double* H = (double*)calloc(HNETN, sizeof(double));
    compact_to_hnet(pu, pv, Hc, H);
    rsurf_hermite(pu, pv, H, R);
    free(H);
    return ORC_OK;
}
double orc_rsurf_bound2(int pu, int pv, const double* Hc, const double* R)
{
    double* H = (double*)calloc(HNETN, sizeof(double));
    compact_to_hnet(pu, pv, Hc, H);
    double b = rsurf_bound2(pu, pv, H, R);
    free(H);
    return b;
}

/* (w: NULL, or the weights of every control point of the set; a surface
 * whose weights are all equal takes the non-rational route) */
static int64_t decompose_one_surface(int64_t s, const int32_t* pu_, const int32_t* pv_, const int32_t* nu_,
                                     const int32_t* nv_, const int64_t* kuoff, const double* ku,
                                     const int64_t* kvoff, const double* kv, const int64_t* coff,
                                     const double* cps, const double* w, double tol_rel, int64_t first,
                                     int64_t cap, double* ctrl, double* prange, int* maxdepth, int* notconv)
{
    int pu = pu_[s], pv = pv_[s], nu = nu_[s], nv = nv_[s];
    if (pu > SMAXP || pv > SMAXP) return -1;
    const double* U = ku + kuoff[s];
    const double* V = kv + kvoff[s];
    const double* P = cps + 3 * coff[s];
    if (coff[s + 1] - coff[s] != (int64_t)nu * nv) return -1;
    if (!check_knots(pu, U, kuoff[s + 1] - kuoff[s], nu)) return -1;
    if (!check_knots(pv, V, kvoff[s + 1] - kvoff[s], nv)) return -1;
    for (int64_t i = 0; i < 3 * (int64_t)nu * nv; ++i) if (!isfinite(P[i])) return -1;
    const double* ws = w ? w + coff[s] : NULL;
    int rat = ws ? weights_kind(ws, (int64_t)nu * nv) : 0;
    if (rat < 0) return -1;
    double thr = tol_rel * box_diag(P, (int64_t)nu * nv);
    surf_ctx X;
    X.pu = pu; X.pv = pv; X.thr2 = thr * thr; X.cap = cap; X.ctrl = ctrl; X.prange = prange;
    X.count = first; X.maxdepth = 0; X.notconv = 0;
    double* Q = (double*)malloc(sizeof(double) * (rat ? HNETN : NETN));
    double *wP = NULL, *w3 = NULL;
    if (rat) {
        int64_t np = (int64_t)nu * nv;
        wP = (double*)malloc(sizeof(double) * 3 * (size_t)np);
        w3 = (double*)malloc(sizeof(double) * 3 * (size_t)np);
        for (int64_t i = 0; i < np; ++i) {
            for (int c = 0; c < 3; ++c) wP[3 * i + c] = ws[i] * P[3 * i + c];
            w3[3 * i] = ws[i];
            w3[3 * i + 1] = 0.0;
            w3[3 * i + 2] = 0.0;
        }
    }
    for (int qu = pu; qu <= nu - 1; ++qu) {
        if (!(U[qu] < U[qu + 1])) continue;
        for (int qv = pv; qv <= nv - 1; ++qv) {
            if (!(V[qv] < V[qv + 1])) continue;
            X.u0 = U[qu]; X.u1 = U[qu + 1]; X.v0 = V[qv]; X.v1 = V[qv + 1];
            X.span_first = X.count;
            if (rat) {
                rsurf_span_bezier(pu, pv, U, qu, V, qv, wP, w3, nv, Q);
                rsurf_node(&X, Q, 0, 0, 0, 0);
            } else {
                surf_span_bezier(pu, pv, U, qu, V, qv, P, nv, Q);
                surf_node(&X, Q, 0, 0, 0, 0);
            }
        }
    }
    free(Q);
    free(wP);
    free(w3);
    *maxdepth = X.maxdepth;
    *notconv = X.notconv;
    return X.count - first;
}

int orc_decompose_surfaces(int64_t n, const int32_t* pu_, const int32_t* pv_, const int32_t* nu_,
                           const int32_t* nv_, const int64_t* kuoff, const double* ku,
                           const int64_t* kvoff, const double* kv, const int64_t* coff,
                           const double* cps, const double* w, double tol_rel, int64_t* seg_off, int64_t cap,
                           double* ctrl, double* prange, int64_t* total, int* maxdepth)
{
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int md = 0, nc = 0, bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : md) reduction(| : nc, bad)
    for (int64_t s = 0; s < n; ++s) {
        int m1 = 0, n1 = 0;
        cnt[s] = decompose_one_surface(s, pu_, pv_, nu_, nv_, kuoff, ku, kvoff, kv, coff, cps, w, tol_rel, 0, 0,
                                       NULL, NULL, &m1, &n1);
        if (cnt[s] < 0) bad = 1;
        if (m1 > md) md = m1;
        nc |= n1;
    }
    if (bad) { free(cnt); return ORC_EINVAL; }
    seg_off[0] = 0;
    for (int64_t s = 0; s < n; ++s) seg_off[s + 1] = seg_off[s] + cnt[s];
    int64_t tot = seg_off[n];
    if (ctrl && tot <= cap) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t s = 0; s < n; ++s) {
            int m1, n1;
            decompose_one_surface(s, pu_, pv_, nu_, nv_, kuoff, ku, kvoff, kv, coff, cps, w, tol_rel, seg_off[s], cap,
                                  ctrl, prange, &m1, &n1);
        }
    }
    free(cnt);
    *total = tot;
    if (maxdepth) *maxdepth = md;
    if (nc) return ORC_ENOTCONV;
    return tot <= cap ? ORC_OK : ORC_ENOSPACE;
}

/* ------------------------------------------------------------------ */
/* projection / inversion on the original curve (Sec. 3)                */
/* ------------------------------------------------------------------ */

#define OSAMP 64 /* samples per non-empty span */

typedef struct {
    int p, m;
    const double* U;
    const double* P;
    const double* w; /* NULL: non-rational */
    const double* q;
} curve_prob;

/* D = |C - q|^2, E = D', Ep = E' (Eqs. Dt, Et, E't) */
static void dist_ders(const curve_prob* B, double t, double* D, double* E, double* Ep)
{
    double C[3], C1[3], C2[3];
    curve_eval(B->p, B->U, B->m, B->P, B->w, t, C, C1, C2);
    double d[3] = { C[0] - B->q[0], C[1] - B->q[1], C[2] - B->q[2] };
    *D = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (E) *E = 2.0 * (d[0] * C1[0] + d[1] * C1[1] + d[2] * C1[2]);
    if (Ep) *Ep = 2.0 * ((C1[0] * C1[0] + C1[1] * C1[1] + C1[2] * C1[2]) +
                         (d[0] * C2[0] + d[1] * C2[1] + d[2] * C2[2]));
}

/* safeguarded Newton for a minimum of D in [lo, hi] from t0: a Newton step on
 * E when E' > 0 and the step stays inside the bracket, bisection otherwise;
 * the bracket keeps the side on which D descends. */
static double newton_min_1d(const curve_prob* B, double lo, double hi, double t0, double eps)
{
    double t = t0;
    for (int it = 0; it < 100; ++it) {
        double D, E, Ep;
        dist_ders(B, t, &D, &E, &Ep);
        if (E > 0.0) hi = t;
        else if (E < 0.0) lo = t;
        else break;
        double tn = (Ep > 0.0) ? t - E / Ep : 0.5 * (lo + hi);
        if (!(tn >= lo && tn <= hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= eps || hi - lo <= eps) { t = tn; break; }
        t = tn;
    }
    return t;
}

/* bounds of |C'(t)| and |C''(t)| on span q.  The derivatives are B-splines
 * with control points D1_i = p (P_i - P_{i-1})/(t_{i+p} - t_i) and
 * D2_i = (p-1)(D1_i - D1_{i-1})/(t_{i+p-1} - t_i); B-spline weights are a
 * convex partition of unity, so the largest control-point norm bounds each. */
static void curve_deriv_bounds(int p, const double* U, const double* P, int q, double* V, double* A)
{
    double D1[ONP + 1][3];
    double v = 0.0, a = 0.0;
    for (int i = q - p + 1; i <= q; ++i) {
        int r = i - (q - p + 1);
        double den = U[i + p] - U[i];
        for (int c = 0; c < 3; ++c) D1[r][c] = den != 0.0 ? p * (P[3 * i + c] - P[3 * (i - 1) + c]) / den : 0.0;
        double w = sqrt(D1[r][0] * D1[r][0] + D1[r][1] * D1[r][1] + D1[r][2] * D1[r][2]);
        if (w > v) v = w;
    }
    for (int i = q - p + 2; i <= q; ++i) {
        int r = i - (q - p + 1);
        double den = U[i + p - 1] - U[i];
        if (den == 0.0) continue;
        double x[3];
        for (int c = 0; c < 3; ++c) x[c] = (p - 1) * (D1[r][c] - D1[r - 1][c]) / den;
        double w = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (w > a) a = w;
    }
    *V = v;
    *A = a;
}

/* the same bounds on span q of a rational curve C = A/W.  With the span's
 * points taken relative to P_r = P_{q-p} (which changes neither derivative),
 * C - P_r = A/W with A = sum N_i w_i (P_i - P_r), and the quotient rule gives
 *   |C'|  <= (|A'| + |W'| r) / w_min,
 *   |C''| <= (|A''| + 2 |W'| |C'| + |W''| r) / w_min,
 * r = max_i |P_i - P_r| (C is a convex combination of the span's points),
 * w_min = min_i w_i (W is one of the weights), and |A'|, |A''|, |W'|, |W''|
 * bounded by the norms of their B-spline control points (the rule above
 * applied to the homogeneous points (w_i (P_i - P_r), w_i)). */
static void rcurve_deriv_bounds(int p, const double* U, const double* P, const double* w, int q, double* V,
                                double* A)
{
    double H[ONP + 1][4], D1[ONP + 1][4];
    const double* Pr = P + 3 * (q - p);
    double r = 0.0, wmin = INFINITY;
    for (int i = q - p; i <= q; ++i) {
        int j = i - (q - p);
        double d[3] = { P[3 * i] - Pr[0], P[3 * i + 1] - Pr[1], P[3 * i + 2] - Pr[2] };
        double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (nd > r) r = nd;
        if (w[i] < wmin) wmin = w[i];
        for (int c = 0; c < 3; ++c) H[j][c] = w[i] * d[c];
        H[j][3] = w[i];
    }
    double a1 = 0.0, w1 = 0.0, a2 = 0.0, w2 = 0.0;
    for (int i = q - p + 1; i <= q; ++i) {
        int j = i - (q - p);
        double den = U[i + p] - U[i];
        for (int c = 0; c < 4; ++c) D1[j][c] = den != 0.0 ? p * (H[j][c] - H[j - 1][c]) / den : 0.0;
        double na = sqrt(D1[j][0] * D1[j][0] + D1[j][1] * D1[j][1] + D1[j][2] * D1[j][2]);
        if (na > a1) a1 = na;
        if (fabs(D1[j][3]) > w1) w1 = fabs(D1[j][3]);
    }
    for (int i = q - p + 2; i <= q; ++i) {
        int j = i - (q - p);
        double den = U[i + p - 1] - U[i];
        if (den == 0.0) continue;
        double x[4];
        for (int c = 0; c < 4; ++c) x[c] = (p - 1) * (D1[j][c] - D1[j - 1][c]) / den;
        double na = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (na > a2) a2 = na;
        if (fabs(x[3]) > w2) w2 = fabs(x[3]);
    }
    *V = (a1 + w1 * r) / wmin;
    *A = (a2 + 2.0 * w1 * *V + w2 * r) / wmin;
}

/* exported for the pins: V, A on span q (w NULL: non-rational) */
int orc_curve_deriv_bounds(int p, const double* U, int64_t nU, const double* P, const double* w, int q, double* V,
                           double* A)
{
    if (p < 1 || p > OMAXP || q < p || q >= nU - p - 1 || !(U[q] < U[q + 1])) return ORC_EINVAL;
    if (w) rcurve_deriv_bounds(p, U, P, w, q, V, A);
    else curve_deriv_bounds(p, U, P, q, V, A);
    return ORC_OK;
}

typedef struct { double a, b, Da, Db; int depth; } ival_t;

/* lower bound of D = |C-q|^2 on [a,b] inside one span (C polynomial there):
 * first order: |C-q| >= (d_a + d_b - V h)/2;
 * second order: D >= min(D_a, D_b) - h^2/8 max|D''|,
 * with |D''| = 2|C'.C' + (C-q).C''| <= 2 (V^2 + (max(d_a,d_b) + V h/2) A). */
static double ival_lower_bound(const ival_t* iv, double V, double A)
{
    double h = iv->b - iv->a, da = sqrt(iv->Da), db = sqrt(iv->Db);
    double l1 = 0.5 * (da + db - V * h);
    l1 = l1 > 0.0 ? l1 * l1 : 0.0;
    double K = 2.0 * (V * V + ((da > db ? da : db) + 0.5 * V * h) * A);
    double l2 = (iv->Da < iv->Db ? iv->Da : iv->Db) - 0.125 * h * h * K;
    return l1 > l2 ? l1 : l2;
}

/* global minimiser of |C(t) - q| over [t_p, t_{m+1}]:
 *  1. dense sampling (OSAMP per non-empty span plus all span ends) and one
 *     safeguarded Newton per sampled basin, plus every knot as a candidate;
 *  2. branch and bound over the sample intervals with the rigorous lower
 *     bound above: an interval whose bound is below the best distance found is
 *     bisected (its midpoint evaluated, and polished by Newton when it is a
 *     local minimum) until the bound clears the best or the interval is
 *     2^-44 of its sample step.  No basin can therefore hide between samples. */
static void project_curve_one(int p, const double* U, int m, const double* P, const double* w, const double* q,
                              double* t_out, double* d_out)
{
    curve_prob B = { p, m, U, P, w, q };
    int ns = 0;
    for (int k = p; k <= m; ++k) if (U[k] < U[k + 1]) ++ns;
    int nsamp = ns * OSAMP + 1;
    double* ts = (double*)malloc(sizeof(double) * (size_t)nsamp);
    double* Ds = (double*)malloc(sizeof(double) * (size_t)nsamp);
    double* Vs = (double*)malloc(sizeof(double) * (size_t)nsamp);
    double* As = (double*)malloc(sizeof(double) * (size_t)nsamp);
    int j = 0;
    double tlast = 0.0;
    for (int k = p; k <= m; ++k) {
        if (!(U[k] < U[k + 1])) continue;
        double V, A;
        if (w) rcurve_deriv_bounds(p, U, P, w, k, &V, &A);
        else curve_deriv_bounds(p, U, P, k, &V, &A);
        for (int s = 0; s < OSAMP; ++s) {
            Vs[j] = V;
            As[j] = A;
            ts[j++] = U[k] + (U[k + 1] - U[k]) * ((double)s / OSAMP);
        }
        tlast = U[k + 1];
    }
    ts[j++] = tlast;
    double t0 = ts[0], t1 = tlast, eps = 1e-15 * (t1 - t0);
    for (int i = 0; i < nsamp; ++i) dist_ders(&B, ts[i], &Ds[i], NULL, NULL);
    double bestD = INFINITY, bestT = t0;
#define CONSIDER(tt)                                                          \
    do {                                                                      \
        double D_;                                                            \
        dist_ders(&B, (tt), &D_, NULL, NULL);                                 \
        if (D_ < bestD || (D_ == bestD && (tt) < bestT)) { bestD = D_; bestT = (tt); } \
    } while (0)
    for (int i = 0; i < nsamp; ++i) {
        int lmin = (i == 0 || Ds[i] <= Ds[i - 1]) && (i == nsamp - 1 || Ds[i] <= Ds[i + 1]);
        if (!lmin) continue;
        double lo = ts[i > 0 ? i - 1 : 0], hi = ts[i < nsamp - 1 ? i + 1 : nsamp - 1];
        double tn = newton_min_1d(&B, lo, hi, ts[i], eps);
        CONSIDER(tn);
        CONSIDER(ts[i]);
    }
    for (int k = p; k <= m + 1; ++k) {
        if (U[k] < t0 || U[k] > t1) continue;
        CONSIDER(U[k]);
    }
    /* branch and bound, depth-first with an explicit stack */
    int cap = 256, top = 0;
    ival_t* st = (ival_t*)malloc(sizeof(ival_t) * (size_t)cap);
    for (int i = 0; i + 1 < nsamp; ++i) {
        double V = Vs[i], A = As[i];
        st[top++] = (ival_t){ ts[i], ts[i + 1], Ds[i], Ds[i + 1], 0 };
        while (top > 0) {
            ival_t iv = st[--top];
            if (iv.depth >= 44 || !(ival_lower_bound(&iv, V, A) < bestD)) continue;
            double mid = 0.5 * (iv.a + iv.b), Dm;
            dist_ders(&B, mid, &Dm, NULL, NULL);
            if (Dm < bestD || (Dm == bestD && mid < bestT)) { bestD = Dm; bestT = mid; }
            if (Dm <= iv.Da && Dm <= iv.Db) {
                double tn = newton_min_1d(&B, iv.a, iv.b, mid, eps);
                CONSIDER(tn);
            }
            if (top + 2 > cap) { cap *= 2; st = (ival_t*)realloc(st, sizeof(ival_t) * (size_t)cap); }
            st[top++] = (ival_t){ mid, iv.b, Dm, iv.Db, iv.depth + 1 };
            st[top++] = (ival_t){ iv.a, mid, iv.Da, Dm, iv.depth + 1 };
        }
    }
    free(st);
#undef CONSIDER
    *t_out = bestT;
    *d_out = sqrt(bestD);
    free(ts); free(Ds); free(Vs); free(As);
}

/* w: NULL (non-rational) or the weights of every control point of the set */
int orc_project_curves(int64_t n, const int32_t* deg, const int64_t* koff, const double* knots,
                       const int64_t* coff, const double* cps, const double* w, int64_t nq, const int32_t* qc,
                       const double* qxyz, double* t_out, double* d_out, int nthreads)
{
    for (int64_t k = 0; k < nq; ++k)
        if (qc[k] < 0 || qc[k] >= n) return ORC_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nq; ++k) {
        int64_t c = qc[k];
        int m = (int)(coff[c + 1] - coff[c]) - 1;
        project_curve_one(deg[c], knots + koff[c], m, cps + 3 * coff[c], w ? w + coff[c] : NULL, qxyz + 3 * k,
                          &t_out[k], &d_out[k]);
    }
    return ORC_OK;
}

/* threads the OpenMP runtime would use */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* projection / inversion on the original surface                       */
/* ------------------------------------------------------------------ */

#define OSAMP2 16 /* samples per span and direction */

typedef struct {
    int pu, pv, mu, mv, nv;
    const double* U;
    const double* V;
    const double* P;
    const double* q;
    const double* w; /* NULL: non-rational */
} surf_prob;

static double sdist(const surf_prob* B, double u, double v, double* g, double* H)
{
    double o[18];
    surface_eval(B->pu, B->pv, B->U, B->mu, B->V, B->mv, B->P, B->w, B->nv, u, v, o);
    double d[3] = { o[0] - B->q[0], o[1] - B->q[1], o[2] - B->q[2] };
    double D = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (g) {
        const double *Su = o + 3, *Sv = o + 6, *Suu = o + 9, *Suv = o + 12, *Svv = o + 15;
        g[0] = 2.0 * (d[0] * Su[0] + d[1] * Su[1] + d[2] * Su[2]);
        g[1] = 2.0 * (d[0] * Sv[0] + d[1] * Sv[1] + d[2] * Sv[2]);
        H[0] = 2.0 * ((Su[0] * Su[0] + Su[1] * Su[1] + Su[2] * Su[2]) + (d[0] * Suu[0] + d[1] * Suu[1] + d[2] * Suu[2]));
        H[1] = 2.0 * ((Su[0] * Sv[0] + Su[1] * Sv[1] + Su[2] * Sv[2]) + (d[0] * Suv[0] + d[1] * Suv[1] + d[2] * Suv[2]));
        H[2] = 2.0 * ((Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]) + (d[0] * Svv[0] + d[1] * Svv[1] + d[2] * Svv[2]));
    }
    return D;
}

/* 1D problem along an iso-curve of the surface (fixed u or fixed v) */
typedef struct {
    const surf_prob* S;
    int fixu;     /* 1: u fixed = c, parameter is v; 0: v fixed */
    double c;
} iso_prob;

static void iso_ders(const iso_prob* I, double t, double* D, double* E, double* Ep)
{
    double g[2], H[3];
    double u = I->fixu ? I->c : t, v = I->fixu ? t : I->c;
    *D = sdist(I->S, u, v, g, H);
    if (E) *E = I->fixu ? g[1] : g[0];
    if (Ep) *Ep = I->fixu ? H[2] : H[0];
}

static double iso_newton(const iso_prob* I, double lo, double hi, double t0, double eps)
{
    double t = t0;
    for (int it = 0; it < 100; ++it) {
        double D, E, Ep;
        iso_ders(I, t, &D, &E, &Ep);
        if (E > 0.0) hi = t;
        else if (E < 0.0) lo = t;
        else break;
        double tn = (Ep > 0.0) ? t - E / Ep : 0.5 * (lo + hi);
        if (!(tn >= lo && tn <= hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) <= eps || hi - lo <= eps) { t = tn; break; }
        t = tn;
    }
    return t;
}

/* sample parameters of one direction: OSAMP2 per non-empty span plus the end */
static int dir_samples(const double* U, int p, int m, double* out)
{
    int j = 0;
    double last = 0.0;
    for (int k = p; k <= m; ++k) {
        if (!(U[k] < U[k + 1])) continue;
        for (int s = 0; s < OSAMP2; ++s) out[j++] = U[k] + (U[k + 1] - U[k]) * ((double)s / OSAMP2);
        last = U[k + 1];
    }
    out[j++] = last;
    return j;
}

/* bounds of |S_u|, |S_v|, |S_uu|, |S_vv| on span pair (qu, qv) from the
 * derivative control nets (convex partition of unity, as for curves) */
static void surf_deriv_bounds(const surf_prob* B, int qu, int qv, double* Vu, double* Vv, double* Auu,
                              double* Avv)
{
    int pu = B->pu, pv = B->pv;
    const double* U = B->U;
    const double* V = B->V;
    double vu = 0, vv = 0, au = 0, av = 0;
#define PT(i, j) (B->P + 3 * ((int64_t)(i) * B->nv + (j)))
    for (int j = qv - pv; j <= qv; ++j) {
        double D1[SNP][3];
        for (int i = qu - pu + 1; i <= qu; ++i) {
            int r = i - (qu - pu + 1);
            double den = U[i + pu] - U[i];
            for (int c = 0; c < 3; ++c) D1[r][c] = den != 0.0 ? pu * (PT(i, j)[c] - PT(i - 1, j)[c]) / den : 0.0;
            double w = sqrt(D1[r][0] * D1[r][0] + D1[r][1] * D1[r][1] + D1[r][2] * D1[r][2]);
            if (w > vu) vu = w;
        }
        for (int i = qu - pu + 2; i <= qu; ++i) {
            int r = i - (qu - pu + 1);
            double den = U[i + pu - 1] - U[i];
            if (den == 0.0) continue;
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = (pu - 1) * (D1[r][c] - D1[r - 1][c]) / den;
            double w = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            if (w > au) au = w;
        }
    }
    for (int i = qu - pu; i <= qu; ++i) {
        double D1[SNP][3];
        for (int j = qv - pv + 1; j <= qv; ++j) {
            int r = j - (qv - pv + 1);
            double den = V[j + pv] - V[j];
            for (int c = 0; c < 3; ++c) D1[r][c] = den != 0.0 ? pv * (PT(i, j)[c] - PT(i, j - 1)[c]) / den : 0.0;
            double w = sqrt(D1[r][0] * D1[r][0] + D1[r][1] * D1[r][1] + D1[r][2] * D1[r][2]);
            if (w > vv) vv = w;
        }
        for (int j = qv - pv + 2; j <= qv; ++j) {
            int r = j - (qv - pv + 1);
            double den = V[j + pv - 1] - V[j];
            if (den == 0.0) continue;
            double x[3];
            for (int c = 0; c < 3; ++c) x[c] = (pv - 1) * (D1[r][c] - D1[r - 1][c]) / den;
            double w = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            if (w > av) av = w;
        }
    }
#undef PT
    *Vu = vu; *Vv = vv; *Auu = au; *Avv = av;
}

/* the same bounds for a rational surface S = A/W on span pair (qu, qv):
 * with the span pair's points relative to P_r = P_{qu-pu, qv-pv} (which
 * changes no derivative), S - P_r = A/W with A = sum N w (P - P_r), and the
 * quotient rule gives, along u (v alike),
 *   |S_u|  <= (|A_u| + |W_u| r) / w_min,
 *   |S_uu| <= (|A_uu| + 2 |W_u| |S_u| + |W_uu| r) / w_min,
 * r = max |P - P_r| over the span pair's points (S is a convex combination
 * of them), w_min their smallest weight, and |A_u|, |A_uu|, |W_u|, |W_uu|
 * bounded by the norms of the derivative control nets of the homogeneous
 * points (w (P - P_r), w), as in surf_deriv_bounds. */
static void rsurf_deriv_bounds(const surf_prob* B, int qu, int qv, double* Vu, double* Vv, double* Auu,
                               double* Avv)
{
    int pu = B->pu, pv = B->pv;
    const double* U = B->U;
    const double* V = B->V;
#define PT(i, j) (B->P + 3 * ((int64_t)(i) * B->nv + (j)))
#define WT(i, j) (B->w[(int64_t)(i) * B->nv + (j)])
    const double* Pr = PT(qu - pu, qv - pv);
    double r = 0.0, wmin = INFINITY;
    for (int i = qu - pu; i <= qu; ++i)
        for (int j = qv - pv; j <= qv; ++j) {
            double d[3] = { PT(i, j)[0] - Pr[0], PT(i, j)[1] - Pr[1], PT(i, j)[2] - Pr[2] };
            double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (nd > r) r = nd;
            if (WT(i, j) < wmin) wmin = WT(i, j);
        }
    /* a1/w1: first derivative net norms (numerator / weight), a2/w2: second;
     * index 0 along u, 1 along v */
    double a1[2] = { 0, 0 }, w1[2] = { 0, 0 }, a2[2] = { 0, 0 }, w2[2] = { 0, 0 };
    for (int dir = 0; dir < 2; ++dir) {
        int p = dir == 0 ? pu : pv, q = dir == 0 ? qu : qv;
        const double* K = dir == 0 ? U : V;
        int olo = dir == 0 ? qv - pv : qu - pu, ohi = dir == 0 ? qv : qu;
        for (int o = olo; o <= ohi; ++o) {
            double H[SNP][4], D1[SNP][4];
            for (int i = q - p; i <= q; ++i) {
                int ii = dir == 0 ? i : o, jj = dir == 0 ? o : i;
                double wij = WT(ii, jj);
                for (int c = 0; c < 3; ++c) H[i - (q - p)][c] = wij * (PT(ii, jj)[c] - Pr[c]);
                H[i - (q - p)][3] = wij;
            }
            for (int i = q - p + 1; i <= q; ++i) {
                int k = i - (q - p);
                double den = K[i + p] - K[i];
                for (int c = 0; c < 4; ++c) D1[k][c] = den != 0.0 ? p * (H[k][c] - H[k - 1][c]) / den : 0.0;
                double na = sqrt(D1[k][0] * D1[k][0] + D1[k][1] * D1[k][1] + D1[k][2] * D1[k][2]);
                if (na > a1[dir]) a1[dir] = na;
                if (fabs(D1[k][3]) > w1[dir]) w1[dir] = fabs(D1[k][3]);
            }
            for (int i = q - p + 2; i <= q; ++i) {
                int k = i - (q - p);
                double den = K[i + p - 1] - K[i];
                if (den == 0.0) continue;
                double x[4];
                for (int c = 0; c < 4; ++c) x[c] = (p - 1) * (D1[k][c] - D1[k - 1][c]) / den;
                double na = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                if (na > a2[dir]) a2[dir] = na;
                if (fabs(x[3]) > w2[dir]) w2[dir] = fabs(x[3]);
            }
        }
    }
#undef PT
#undef WT
    *Vu = (a1[0] + w1[0] * r) / wmin;
    *Vv = (a1[1] + w1[1] * r) / wmin;
    *Auu = (a2[0] + 2.0 * w1[0] * *Vu + w2[0] * r) / wmin;
    *Avv = (a2[1] + 2.0 * w1[1] * *Vv + w2[1] * r) / wmin;
}

typedef struct { double u0, u1, v0, v1, D[4]; int depth; } cell_t; /* D: (u0,v0),(u1,v0),(u0,v1),(u1,v1) */

/* lower bound of D on a cell inside one span pair (S polynomial there):
 * first order: d >= min corner d - (Vu hu + Vv hv)/2;
 * second order: bilinear interpolation error, D >= min corner D
 *   - (hu^2 |D_uu| + hv^2 |D_vv|)/8, |D_uu| <= 2 (Vu^2 + R Auu), R the
 *   largest distance on the cell. */
static double cell_lower_bound(const cell_t* c, double Vu, double Vv, double Au, double Av)
{
    double hu = c->u1 - c->u0, hv = c->v1 - c->v0;
    double Dmin = c->D[0], Dmax = c->D[0];
    for (int k = 1; k < 4; ++k) {
        if (c->D[k] < Dmin) Dmin = c->D[k];
        if (c->D[k] > Dmax) Dmax = c->D[k];
    }
    double reach = 0.5 * (Vu * hu + Vv * hv);
    double l1 = sqrt(Dmin) - reach;
    l1 = l1 > 0.0 ? l1 * l1 : 0.0;
    double R = sqrt(Dmax) + reach;
    double l2 = Dmin - 0.125 * (hu * hu * 2.0 * (Vu * Vu + R * Au) + hv * hv * 2.0 * (Vv * Vv + R * Av));
    return l1 > l2 ? l1 : l2;
}

/* damped, domain-clamped Newton on grad D from (u,v); returns the end point */
static void surf_polish(const surf_prob* B, double ua, double ub, double va, double vb, double* pu_,
                        double* pv_, double eps)
{
    double u = *pu_, v = *pv_;
    for (int it = 0; it < 100; ++it) {
        double g[2], H[3];
        double D = sdist(B, u, v, g, H);
        double det = H[0] * H[2] - H[1] * H[1];
        double su, sv;
        if (H[0] > 0.0 && det > 0.0) {
            su = -(H[2] * g[0] - H[1] * g[1]) / det;
            sv = -(H[0] * g[1] - H[1] * g[0]) / det;
        } else {
            double gn = sqrt(g[0] * g[0] + g[1] * g[1]);
            if (gn == 0.0) break;
            su = -g[0] / gn * (ub - ua) * (1.0 / 64);
            sv = -g[1] / gn * (vb - va) * (1.0 / 64);
        }
        double lam = 1.0, un = u, vn = v, Dn = D;
        int ok = 0;
        for (int ls = 0; ls < 40; ++ls) {
            un = u + lam * su; vn = v + lam * sv;
            if (un < ua) un = ua;
            if (un > ub) un = ub;
            if (vn < va) vn = va;
            if (vn > vb) vn = vb;
            Dn = sdist(B, un, vn, NULL, NULL);
            if (Dn <= D) { ok = 1; break; }
            lam *= 0.5;
        }
        if (!ok) break;
        double step = fabs(un - u) + fabs(vn - v);
        u = un; v = vn;
        if (step <= eps) break;
    }
    *pu_ = u; *pv_ = v;
}

static void project_surface_one(const surf_prob* B, double* uv_out, double* d_out)
{
    int nsu_max = (B->mu + 2) * OSAMP2 + 2, nsv_max = (B->mv + 2) * OSAMP2 + 2;
    double* us = (double*)malloc(sizeof(double) * (size_t)nsu_max);
    double* vs = (double*)malloc(sizeof(double) * (size_t)nsv_max);
    int nsu = dir_samples(B->U, B->pu, B->mu, us);
    int nsv = dir_samples(B->V, B->pv, B->mv, vs);
    double* Dg = (double*)malloc(sizeof(double) * (size_t)nsu * (size_t)nsv);
    for (int i = 0; i < nsu; ++i)
        for (int j = 0; j < nsv; ++j) Dg[(int64_t)i * nsv + j] = sdist(B, us[i], vs[j], NULL, NULL);
    double ua = us[0], ub = us[nsu - 1], va = vs[0], vb = vs[nsv - 1];
    double epsu = 1e-15 * (ub - ua), epsv = 1e-15 * (vb - va);
    double bestD = INFINITY, bu = ua, bv = va;
#define CONSIDER2(uu, vv)                                                                \
    do {                                                                                 \
        double D_ = sdist(B, (uu), (vv), NULL, NULL);                                    \
        if (D_ < bestD || (D_ == bestD && ((uu) < bu || ((uu) == bu && (vv) < bv)))) {  \
            bestD = D_; bu = (uu); bv = (vv);                                            \
        }                                                                                \
    } while (0)
    /* interior stationary points: damped Newton on grad D from each sampled
     * basin, kept inside the domain */
    for (int i = 0; i < nsu; ++i) {
        for (int j = 0; j < nsv; ++j) {
            double Dc = Dg[(int64_t)i * nsv + j];
            int lmin = 1;
            for (int di = -1; di <= 1 && lmin; ++di)
                for (int dj = -1; dj <= 1; ++dj) {
                    int a = i + di, b = j + dj;
                    if ((di == 0 && dj == 0) || a < 0 || b < 0 || a >= nsu || b >= nsv) continue;
                    if (Dg[(int64_t)a * nsv + b] < Dc) { lmin = 0; break; }
                }
            if (!lmin) continue;
            CONSIDER2(us[i], vs[j]);
            double u = us[i], v = vs[j];
            surf_polish(B, ua, ub, va, vb, &u, &v, epsu + epsv);
            CONSIDER2(u, v);
        }
    }
    /* boundary and crease iso-curves: the four domain edges and every interior
     * knot line of multiplicity >= degree (where D need not be smooth) */
    int niso = 0;
    double isoc[4096];
    int isofix[4096];
    isoc[niso] = ua; isofix[niso++] = 1;
    isoc[niso] = ub; isofix[niso++] = 1;
    isoc[niso] = va; isofix[niso++] = 0;
    isoc[niso] = vb; isofix[niso++] = 0;
    for (int dir = 0; dir < 2; ++dir) {
        const double* K = dir == 0 ? B->U : B->V;
        int p = dir == 0 ? B->pu : B->pv, m = dir == 0 ? B->mu : B->mv;
        double lo = dir == 0 ? ua : va, hi = dir == 0 ? ub : vb;
        for (int k = p + 1; k <= m; ++k) {
            if (!(K[k] > lo && K[k] < hi) || K[k] == K[k - 1]) continue;
            int mult = 1;
            while (k + mult <= m && K[k + mult] == K[k]) ++mult;
            if (mult >= p && niso < 4096) { isoc[niso] = K[k]; isofix[niso++] = dir == 0 ? 1 : 0; }
        }
    }
    for (int e = 0; e < niso; ++e) {
        iso_prob I = { B, isofix[e], isoc[e] };
        const double* ts = isofix[e] ? vs : us;
        int nt = isofix[e] ? nsv : nsu;
        double eps = isofix[e] ? epsv : epsu;
        double* Dl = (double*)malloc(sizeof(double) * (size_t)nt);
        for (int k = 0; k < nt; ++k) iso_ders(&I, ts[k], &Dl[k], NULL, NULL);
        for (int k = 0; k < nt; ++k) {
            int lmin = (k == 0 || Dl[k] <= Dl[k - 1]) && (k == nt - 1 || Dl[k] <= Dl[k + 1]);
            if (!lmin) continue;
            double lo = ts[k > 0 ? k - 1 : 0], hi = ts[k < nt - 1 ? k + 1 : nt - 1];
            double tn = iso_newton(&I, lo, hi, ts[k], eps);
            if (isofix[e]) { CONSIDER2(isoc[e], tn); CONSIDER2(isoc[e], ts[k]); }
            else { CONSIDER2(tn, isoc[e]); CONSIDER2(ts[k], isoc[e]); }
        }
        free(Dl);
    }
    /* branch and bound over the sample cells of every span pair, with the
     * rigorous bound of cell_lower_bound: a cell whose bound is below the best
     * squared distance is split in four (centre polished by Newton when it is
     * below its corners) until the bound clears or depth 30 is reached */
    {
        int cap = 1024, top = 0;
        cell_t* st = (cell_t*)malloc(sizeof(cell_t) * (size_t)cap);
        int i0 = 0;
        for (int qu = B->pu; qu <= B->mu; ++qu) {
            if (!(B->U[qu] < B->U[qu + 1])) continue;
            int j0 = 0;
            for (int qv = B->pv; qv <= B->mv; ++qv) {
                if (!(B->V[qv] < B->V[qv + 1])) continue;
                double Vu, Vv, Au, Av;
                if (B->w) rsurf_deriv_bounds(B, qu, qv, &Vu, &Vv, &Au, &Av);
                else surf_deriv_bounds(B, qu, qv, &Vu, &Vv, &Au, &Av);
                for (int a = 0; a < OSAMP2; ++a)
                    for (int b = 0; b < OSAMP2; ++b) {
                        int i = i0 + a, jj = j0 + b;
                        cell_t c0 = { us[i], us[i + 1], vs[jj], vs[jj + 1],
                                      { Dg[(int64_t)i * nsv + jj], Dg[(int64_t)(i + 1) * nsv + jj],
                                        Dg[(int64_t)i * nsv + jj + 1], Dg[(int64_t)(i + 1) * nsv + jj + 1] },
                                      0 };
                        st[top++] = c0;
                        while (top > 0) {
                            cell_t c = st[--top];
                            if (c.depth >= 30 || !(cell_lower_bound(&c, Vu, Vv, Au, Av) < bestD)) continue;
                            double um = 0.5 * (c.u0 + c.u1), vm = 0.5 * (c.v0 + c.v1);
                            double Dmid[5] = { sdist(B, um, c.v0, NULL, NULL), sdist(B, c.u0, vm, NULL, NULL),
                                               sdist(B, um, vm, NULL, NULL), sdist(B, c.u1, vm, NULL, NULL),
                                               sdist(B, um, c.v1, NULL, NULL) };
                            double pu5[5] = { um, c.u0, um, c.u1, um }, pv5[5] = { c.v0, vm, vm, vm, c.v1 };
                            for (int k = 0; k < 5; ++k)
                                if (Dmid[k] < bestD) { bestD = Dmid[k]; bu = pu5[k]; bv = pv5[k]; }
                            if (Dmid[2] <= c.D[0] && Dmid[2] <= c.D[1] && Dmid[2] <= c.D[2] && Dmid[2] <= c.D[3]) {
                                double u = um, v = vm;
                                surf_polish(B, ua, ub, va, vb, &u, &v, epsu + epsv);
                                CONSIDER2(u, v);
                            }
                            if (top + 4 > cap) { cap *= 2; st = (cell_t*)realloc(st, sizeof(cell_t) * (size_t)cap); }
                            int d1 = c.depth + 1;
                            st[top++] = (cell_t){ um, c.u1, vm, c.v1, { Dmid[2], Dmid[3], Dmid[4], c.D[3] }, d1 };
                            st[top++] = (cell_t){ c.u0, um, vm, c.v1, { Dmid[1], Dmid[2], c.D[2], Dmid[4] }, d1 };
                            st[top++] = (cell_t){ um, c.u1, c.v0, vm, { Dmid[0], c.D[1], Dmid[2], Dmid[3] }, d1 };
                            st[top++] = (cell_t){ c.u0, um, c.v0, vm, { c.D[0], Dmid[0], Dmid[1], Dmid[2] }, d1 };
                        }
                    }
                j0 += OSAMP2;
            }
            i0 += OSAMP2;
        }
        free(st);
    }
#undef CONSIDER2
    uv_out[0] = bu;
    uv_out[1] = bv;
    *d_out = sqrt(bestD);
    free(us); free(vs); free(Dg);
}

/* w: NULL (non-rational) or the weights of every control point of the set */
int orc_project_surfaces(int64_t n, const int32_t* pu, const int32_t* pv, const int32_t* nu,
                         const int32_t* nv, const int64_t* kuoff, const double* ku,
                         const int64_t* kvoff, const double* kv, const int64_t* coff,
                         const double* cps, const double* w, int64_t nq, const int32_t* qs, const double* qxyz,
                         double* uv_out, double* d_out, int nthreads)
{
    for (int64_t k = 0; k < nq; ++k)
        if (qs[k] < 0 || qs[k] >= n) return ORC_EINVAL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < nq; ++k) {
        int64_t s = qs[k];
        surf_prob B = { pu[s], pv[s], nu[s] - 1, nv[s] - 1, nv[s], ku + kuoff[s], kv + kvoff[s],
                        cps + 3 * coff[s], qxyz + 3 * k, w ? w + coff[s] : NULL };
        project_surface_one(&B, uv_out + 2 * k, &d_out[k]);
    }
    return ORC_OK;
}

/* exported for the pins: the bounds of |S_u|, |S_v|, |S_uu|, |S_vv| on span
 * pair (qu, qv) of one surface (w NULL: non-rational) */
int orc_surf_deriv_bounds(int pu, int pv, const double* U, int nu, const double* V, int nv, const double* P,
                          const double* w, int qu, int qv, double* out /* Vu, Vv, Auu, Avv */)
{
    if (pu < 1 || pv < 1 || pu > SMAXP || pv > SMAXP || qu < pu || qu >= nu || qv < pv || qv >= nv) return ORC_EINVAL;
    surf_prob B = { pu, pv, nu - 1, nv - 1, nv, U, V, P, NULL, w };
    if (w) rsurf_deriv_bounds(&B, qu, qv, out, out + 1, out + 2, out + 3);
    else surf_deriv_bounds(&B, qu, qv, out, out + 1, out + 2, out + 3);
    return ORC_OK;
}
