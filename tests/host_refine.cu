// Host build of the refinement on the original curves (the code the GPU
// runs, csrc/eval.cu), for CPU tests against the oracle at every degree.
#include "../paper_2504_11498_gb300/csrc/eval.cu"

namespace bspl {
// the launcher in eval.cu refers to the query sort, which these host
// entry points never reach
size_t query_ws_bytes(int64_t, int64_t) { return 0; }
cudaError_t sort_by_spline(const int32_t*, int64_t, int64_t, const int32_t*, void*, size_t, int32_t**,
                           unsigned long long**, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace bspl

using namespace bspl;

namespace {
template <int MP, int NC>
void eval_mp(int p, const double* U, int m, const double* P, const double* w, double t, double* C, double* C1,
             double* C2)
{
    SpanCache<MP, NC> S;
    S.q = -1;
    S.rcp = nullptr;
    curve_d2<MP, NC>(U, P, w, p, m, t, S, C, C1, C2);
}

template <int NC>
bool refine_mp(int p, const double* U, int m, const double* P, const double* w, const double* q, int max_iter,
               double& t, double& D, int& n1, int& n2)
{
    if (p <= 7) return refine_one<7, NC>(U, P, w, p, m, q, max_iter, t, D, n1, n2, nullptr);
    if (p <= kEvalMidDeg) return refine_one<kEvalMidDeg, NC>(U, P, w, p, m, q, max_iter, t, D, n1, n2, nullptr);
    return refine_one<kMaxCurveDegree, NC>(U, P, w, p, m, q, max_iter, t, D, n1, n2, nullptr);
}
}  // namespace

extern "C" {

// C, C', C'' of a curve of degree p (knots U, control points P [m+1][3],
// weights w or NULL) at t, through the refinement's evaluation (the instance
// the device uses for that degree)
void hr_eval(int p, const double* U, int m, const double* P, const double* w, double t, double* C, double* C1,
             double* C2)
{
    if (p <= 7) {
        if (w) eval_mp<7, 4>(p, U, m, P, w, t, C, C1, C2);
        else eval_mp<7, 3>(p, U, m, P, w, t, C, C1, C2);
    } else if (p <= kEvalMidDeg) {
        if (w) eval_mp<kEvalMidDeg, 4>(p, U, m, P, w, t, C, C1, C2);
        else eval_mp<kEvalMidDeg, 3>(p, U, m, P, w, t, C, C1, C2);
    } else {
        if (w) eval_mp<kMaxCurveDegree, 4>(p, U, m, P, w, t, C, C1, C2);
        else eval_mp<kMaxCurveDegree, 3>(p, U, m, P, w, t, C, C1, C2);
    }
}

// the refinement of one query from *t: returns whether it converged, with
// the final t, the squared distance and the evaluations made
int hr_refine(int p, const double* U, int m, const double* P, const double* w, const double* q, int max_iter,
              double* t, double* D, int* nev)
{
    int n1 = 0, n2 = 0;
    const bool conv = w ? refine_mp<4>(p, U, m, P, w, q, max_iter, *t, *D, n1, n2)
                        : refine_mp<3>(p, U, m, P, w, q, max_iter, *t, *D, n1, n2);
    *nev = n1 + n2;
    return conv ? 1 : 0;
}
}
