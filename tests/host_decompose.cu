// Host build of the decomposition walk of one surface span pair (the code the
// GPU runs, csrc/decompose.cu), for CPU tests of its bit-exact agreement
// with the oracle.  The block-shared coefficient tables are filled here by
// the same FP64 operations as on the device.
#include "../paper_2504_11498_gb300/csrc/decompose.cu"

namespace bspl {
namespace {
template <int MP>
void host_fill_coef(RedCoef<MP>& cf)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) cf.g33[i][j] = gram_d(3, 3, i, j);
    for (int p = 0; p <= MP; ++p)
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j <= MP; ++j) cf.gp[p][r][j] = j <= p ? gram_d(3, p, 1 + r, j) : 0.0;
    for (int p = 0; p <= MP; ++p) cf.ap[p] = fdiv((double)p, 3.0);
    for (int n = 0; n < MP; ++n)
        for (int i = 0; i <= MP; ++i) {
            cf.ea[n][i] = fdiv((double)i, (double)(n + 1));
            cf.eb[n][i] = fdiv((double)(n + 1 - i), (double)(n + 1));
        }
}
}  // namespace
}  // namespace bspl

using namespace bspl;

// (the device's walk instances: degrees 1..7 (the matrix route), 8..15 and
// 16..31 (the blossom) with the block's coefficient tables, 32..63 (the
// blossom) with the coefficients computed inline)
template <int MP, class CF>
int64_t curve_span(int p, const double* U, int q, const double* P, const double* w, double thr2, double* ctrl,
                   double* prange, int64_t cap, int* err, const CF& cf)
{
    const double* Pl = P + 3 * (q - p);
    CurveLeafOut none{};
    const int64_t n = w ? walk_span_rcurve<MP, false>(p, U, q, Pl, w + (q - p), thr2, 0, none, err, cf)
                        : walk_span_curve<MP, false>(p, U, q, Pl, thr2, 0, none, err, cf);
    if (n > cap) return n;
    CurveLeafOut out{ ctrl, prange };
    if (w) walk_span_rcurve<MP, true>(p, U, q, Pl, w + (q - p), thr2, 0, out, err, cf);
    else walk_span_curve<MP, true>(p, U, q, Pl, thr2, 0, out, err, cf);
    return n;
}

extern "C" {

// box diagonal of a control net, as the device computes it
double hd_box_diag(const double* P, int64_t np) { return box_diag_d(P, np); }

// leaves of span pair (qu, qv) of a surface with degrees (pu, pv), knots U, V
// and net P [n_u][n_v][3]; writes up to cap leaves (ctrl [48], prange [4])
// and returns their count (the count is returned even when above cap)
int64_t hd_surface_span(int pu, int pv, const double* U, int nu, int qu, const double* V, int qv, const double* P,
                        int nv,
                        double tol_rel, double diag, double* ctrl, double* prange, int64_t cap, int* err)
{
    static SurfCoef cf;
    static bool filled = false;
    if (!filled) {
        host_fill_coef<kMaxSurfDegree>(cf);
        filled = true;
    }
    const double thr = tol_rel * diag, thr2 = thr * thr;  // the device computes the same two IEEE products
    *err = 0;
    SurfLeafOut none{};
    const int64_t n = walk_span_surface<false>(pu, pv, U, nu, qu, V, qv, P, nv, thr2, 0, 0, none, err, cf);
    if (n > cap) return n;
    double* rec64 = new double[(size_t)BSPL_SREC64 * (size_t)(n > 0 ? n : 1)];
    float* rec32 = new float[(size_t)BSPL_SREC32 * (size_t)(n > 0 ? n : 1)];
    int64_t* span = new int64_t[(size_t)(n > 0 ? n : 1)];
    double* pbox = new double[4 * (size_t)(n > 0 ? n : 1)];
    double* net = new double[BSPL_SPAN_NET];
    float* net32 = new float[BSPL_SPAN_NET];
    float* pnet = new float[(size_t)BSPL_SPAN_NET * (size_t)(n > 0 ? n : 1)];
    SurfLeafOut out{ ctrl, prange, span, pbox, rec64, rec32, net, net32, pnet };
    walk_span_surface<true>(pu, pv, U, nu, qu, V, qv, P, nv, thr2, 0, 0, out, err, cf);
    delete[] rec64;
    delete[] rec32;
    delete[] span;
    delete[] pbox;
    delete[] net;
    delete[] net32;
    delete[] pnet;
    return n;
}

// leaves of span q of a curve of degree p (knots U, control points P, weights
// w: the rational walk, or the non-rational one when w is NULL): up to cap
// leaves (ctrl [12], prange [2]); returns their count
int64_t hd_curve_span(int p, const double* U, int q, const double* P, const double* w, double tol_rel, double diag,
                      double* ctrl, double* prange, int64_t cap, int* err)
{
    static RedCoef<7> cf7;
    static RedCoef<15> cf15;
    static RedCoef<31> cf31;
    static bool filled = false;
    if (!filled) {
        host_fill_coef<7>(cf7);
        host_fill_coef<15>(cf15);
        host_fill_coef<31>(cf31);
        filled = true;
    }
    const double thr = tol_rel * diag, thr2 = thr * thr;
    *err = 0;
    if (p <= 7) return curve_span<7>(p, U, q, P, w, thr2, ctrl, prange, cap, err, cf7);
    if (p <= 15) return curve_span<15>(p, U, q, P, w, thr2, ctrl, prange, cap, err, cf15);
    if (p <= 31) return curve_span<31>(p, U, q, P, w, thr2, ctrl, prange, cap, err, cf31);
    return curve_span<kMaxCurveDegree>(p, U, q, P, w, thr2, ctrl, prange, cap, err, CoefInline{});
}

// derivative bounds and edge flags the filling walk writes into a patch's
// FP32 record (entries 56..61): the bicubic leaves' records of span pair
// (qu, qv), rec32 [cap][BSPL_SREC32], pbox [cap][4]
int64_t hd_surface_records(int pu, int pv, const double* U, int nu, int qu, const double* V, int qv,
                           const double* P, int nv, double tol_rel, double diag, float* rec32, double* pbox,
                           int64_t cap, int* err)
{
    static SurfCoef cf;
    static bool filled = false;
    if (!filled) {
        host_fill_coef<kMaxSurfDegree>(cf);
        filled = true;
    }
    const double thr = tol_rel * diag, thr2 = thr * thr;
    *err = 0;
    SurfLeafOut none{};
    const int64_t n = walk_span_surface<false>(pu, pv, U, nu, qu, V, qv, P, nv, thr2, 0, 0, none, err, cf);
    if (n > cap) return n;
    const size_t m = (size_t)(n > 0 ? n : 1);
    double* ctrl = new double[48 * m];
    double* prange = new double[4 * m];
    double* rec64 = new double[(size_t)BSPL_SREC64 * m];
    int64_t* span = new int64_t[m];
    double* net = new double[BSPL_SPAN_NET];
    float* net32 = new float[BSPL_SPAN_NET];
    float* pnet = new float[(size_t)BSPL_SPAN_NET * m];
    SurfLeafOut out{ ctrl, prange, span, pbox, rec64, rec32, net, net32, pnet };
    walk_span_surface<true>(pu, pv, U, nu, qu, V, qv, P, nv, thr2, 0, 0, out, err, cf);
    delete[] pnet;
    delete[] ctrl;
    delete[] prange;
    delete[] rec64;
    delete[] span;
    delete[] net;
    delete[] net32;
    return n;
}
}
