// Evaluation of the ORIGINAL B-spline curves and surfaces (Sec. 3, Eq.
// bsplinebasis) at given parameters: one thread per point, span by binary
// search, basis by the triangular Cox-de Boor recursion.  Used to place
// inversion queries on the spline.
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
            const double* U = C.knots + C.knot_off[c];
            double t = fmin(fmax(tq[i], U[p]), U[m + 1]);
            int q = span_of(U, p, m, t);
            double N[kMaxCurveDegree + 1];
            basis<kMaxCurveDegree>(U, q, p, t, N);
            const double* P = C.cps + 3 * C.cp_off[c];
            for (int k = 0; k < 3; ++k) out[k] = 0.0;
            for (int j = 0; j <= p; ++j)
                for (int k = 0; k < 3; ++k) out[k] += N[j] * P[3 * (q - p + j) + k];
        }
    }
    for (int k = 0; k < 3; ++k) xyz[3 * i + k] = out[k];
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

bspl_status eval_surfaces(const bspl_surfaces* c, int64_t n_q, const int32_t* qs, const double* uv, double* xyz,
                          cudaStream_t s)
{
    if (!c || n_q < 0 || (n_q > 0 && (!qs || !uv || !xyz))) return BSPL_EINVAL;
    if (n_q == 0) return BSPL_OK;
    k_eval_surfaces<<<ceil_div(n_q, 128), 128, 0, s>>>(*c, n_q, qs, uv, xyz);
    return cudaGetLastError() == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

}  // namespace bspl
