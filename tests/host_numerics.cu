// Host build of the pure-math helpers the curve query kernels share
// (csrc/query_common.cuh, csrc/clip.cuh), for CPU tests of their decisions:
// the Bernstein form of E and its sign changes, the certified isolation of
// the minima of D on a cubic segment, the two FP64 Newton steps, and the
// paper's search (closed-form quartic roots, elimination, clipping).  Plain C entry
// points over host arrays; no device code runs.
#include "../paper_2504_11498_gb300/csrc/query_common.cuh"
#include "../paper_2504_11498_gb300/csrc/clip.cuh"

using namespace bspl;

extern "C" {

// Bernstein coefficients of E/2 for the local-frame cubic a[12] (q at the
// origin); returns the number of sign changes
int hn_bernstein_f(const float* a, float* b) { return bernstein_E<float>(a, 0.f, 0.f, 0.f, b); }

void hn_end_signs_d(const double* b, int* first, int* last) { end_signs6<double>(b, *first, *last); }

// kind of a pair from its FP32 local-frame cubic (kSeed 0, kEnd0 1, kEnd1 2,
// kEnds 3, kIso 4, kIsoU 5)
int hn_classify(const float* c) { return (int)classify(c); }

// FP32 isolation as the learned path calls it; btol may be null
float hn_isolate_f(const float* a, int maxit, const float* btol, int* uncertain, float* second3)
{
    bool unc = false;
    float u = isolate_min<float>(a, 0.f, 0.f, 0.f, 1e-7f, maxit, second3, btol, btol ? &unc : nullptr);
    if (uncertain) *uncertain = unc ? 1 : 0;
    return u;
}

double hn_isolate_d(const double* a, const double* q, int maxit)
{
    return isolate_min<double>(a, q[0], q[1], q[2], 1e-15, maxit);
}

// the two FP64 steps from u; returns D, writes the final u and the size of
// the second step (1 when it is not converged)
double hn_finish64(const double* a64, const double* q, double* u, double* last)
{
    float a32[9];
    for (int i = 0; i < 9; ++i) a32[i] = (float)a64[3 + i];
    unsigned it = 0;
    return finish64(a64, a32, q, *u, *last, it);
}

// real roots of c[4] x^4 + ... + c[0] (Ferrari)
int hn_quartic_d(const double* c, double* x) { return quartic_roots<double>(c, x); }
int hn_quartic_f(const float* c, float* x) { return quartic_roots<float>(c, x); }

// the paper's search on the FP32 local-frame cubic a[12]
float hn_clip_f(const float* a, float tolE, int rounds, float* second3, int* n_min, int* unsure)
{
    ClipOut o;
    const float u = clip_min<float>(a, tolE, rounds, second3, o);
    *n_min = o.n_min;
    *unsure = o.unsure ? 1 : 0;
    return u;
}
}
