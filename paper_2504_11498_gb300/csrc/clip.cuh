// The paper's own search stage on one (query, segment) pair, as an
// alternative to the seed network and to the sign-variation isolation:
//   * monotone decomposition (Sec. 4.2.3, "Monotonic decomposition"): the
//     roots of E' = dE/du, a quartic, in closed form (Ferrari's method, with
//     the resolvent cubic by Cardano's formula or its trigonometric form),
//     split [0, 1] into pieces on which E is monotone;
//   * elimination (Sec. 4.3, Properties 1 and 2): a piece holds a local
//     minimum of D only when E goes from - to + across it; the segment's
//     ends are minima when E(0) >= 0 or E(1) <= 0;
//   * rebasement and clipping (Sec. 4.3 T matrix; Sec. 4.4.1 Eq.
//     subdivisionmatrix): E on such a piece in Bernstein form, its control
//     polygon's convex hull cut with the axis, the curve clipped to the cut
//     by two de Casteljau subdivisions, until the interval is below 1e-6 of
//     the piece (the paper reports about three rounds); a clip that keeps
//     more than half of the interval is replaced by the half where E
//     changes sign (the usual safeguard of Bezier clipping where E is
//     nearly flat); then the chord's root of the last interval.
// Everything is in the precision R on the local-frame cubic c (C - q with q
// at the origin); host and device.
#pragma once
#include <math.h>

#include "query_common.cuh"

namespace bspl {

// real roots of x^3 + b x^2 + c x + d: the trigonometric form when there are
// three, Cardano's formula when there is one.  Returns their number.
template <class R>
__host__ __device__ inline int cubic_roots(R b, R c, R d, R* x)
{
    const R b3 = b / R(3);
    const R p = c - b * b3;                         // x = y - b/3: y^3 + p y + q
    const R q = d - b3 * c + R(2) * b3 * b3 * b3;
    const R h = q * q / R(4) + p * p * p / R(27);
    if (h > R(0) || p == R(0)) {
        const R sh = sqrt(fmax(h, R(0)));
        x[0] = cbrt(-q / R(2) + sh) + cbrt(-q / R(2) - sh) - b3;
        return 1;
    }
    const R m = R(2) * sqrt(-p / R(3));
    const R th = acos(fmin(fmax(R(3) * q / (p * m), R(-1)), R(1))) / R(3);
    for (int k = 0; k < 3; ++k) x[k] = m * cos(th - R(2.0943951023931953) * R(k)) - b3;
    return 3;
}

// real roots of c4 x^4 + c3 x^3 + c2 x^2 + c1 x + c0 (c[0..4]) by Ferrari's
// method: x = y - b/4 gives y^4 + p y^2 + q y + r; for q != 0 the largest
// root m of the resolvent m^3 + p m^2 + (p^2/4 - r) m - q^2/8 is positive and
// splits it into y^2 -+ s y + (p/2 + m +- q/(2 s)), s = sqrt(2 m); for q = 0
// it is a quadratic in y^2.  A vanishing leading coefficient falls back to
// the cubic (or lower).  Returns the number of roots written (at most 4).
template <class R>
__host__ __device__ inline int quartic_roots(const R* c, R* x)
{
    const R scale = fabs(c[0]) + fabs(c[1]) + fabs(c[2]) + fabs(c[3]) + fabs(c[4]);
    if (!(scale > R(0))) return 0;
    auto quad = [](R b, R c0, R* y) -> int {  // y^2 + b y + c0
        const R disc = b * b - R(4) * c0;
        if (disc < R(0)) return 0;
        const R sq = sqrt(disc);
        // the root of larger magnitude directly, the other from the product
        const R t = R(-0.5) * (b + (b >= R(0) ? sq : -sq));
        if (t == R(0)) {
            y[0] = R(0);
            return 1;
        }
        y[0] = t;
        y[1] = c0 / t;
        return 2;
    };
    if (fabs(c[4]) <= R(1e-7) * scale) {
        if (fabs(c[3]) > R(1e-7) * scale) return cubic_roots(c[2] / c[3], c[1] / c[3], c[0] / c[3], x);
        if (fabs(c[2]) > R(1e-7) * scale) return quad(c[1] / c[2], c[0] / c[2], x);
        if (fabs(c[1]) > R(1e-7) * scale) {
            x[0] = -c[0] / c[1];
            return 1;
        }
        return 0;
    }
    const R b = c[3] / c[4], cc = c[2] / c[4], d = c[1] / c[4], e = c[0] / c[4];
    const R b4 = b / R(4), b2 = b * b;
    const R p = cc - R(0.375) * b2;
    const R q = d - R(0.5) * b * cc + R(0.125) * b2 * b;
    const R r = e - R(0.25) * b * d + R(0.0625) * b2 * cc - R(3.0 / 256.0) * b2 * b2;
    int n = 0;
    R y[4];
    if (fabs(q) <= R(1e-7) * (fabs(p) * (R(1) + fabs(b)) + fabs(r) + R(1e-30))) {
        R z[2];
        const int nz = quad(p, r, z);
        for (int i = 0; i < nz; ++i)
            if (z[i] >= R(0)) {
                const R s = sqrt(z[i]);
                y[n++] = s;
                y[n++] = -s;
            }
    } else {
        R m3[3];
        const int nm = cubic_roots(p, R(0.25) * p * p - r, R(-0.125) * q * q, m3);
        R m = m3[0];
        for (int i = 1; i < nm; ++i) m = fmax(m, m3[i]);
        if (m > R(0)) {
            const R s = sqrt(R(2) * m), w = q / (R(2) * s);
            n += quad(-s, R(0.5) * p + m + w, y + n);
            n += quad(s, R(0.5) * p + m - w, y + n);
        }
    }
    for (int i = 0; i < n; ++i) x[i] = y[i] - b4;
    return n;
}

// power coefficients of E/2 = (C - q).C' (degree 5) for the local-frame cubic
// c[12] (c0 = C(0) - q, c1, c2, c3 by component): e[0..5]
template <class R>
__host__ __device__ inline void power_E(const R* c, R* e)
{
    for (int k = 0; k < 6; ++k) e[k] = R(0);
    for (int k = 0; k < 3; ++k) {
        const R c0 = c[k], c1 = c[3 + k], c2 = c[6 + k], c3 = c[9 + k];
        e[0] += c0 * c1;
        e[1] += R(2) * c0 * c2 + c1 * c1;
        e[2] += R(3) * c0 * c3 + R(3) * c1 * c2;
        e[3] += R(4) * c1 * c3 + R(2) * c2 * c2;
        e[4] += R(5) * c2 * c3;
        e[5] += R(3) * c3 * c3;
    }
}

// de Casteljau of degree-5 Bernstein coefficients at s: keep the left
// ([0, s]) or the right ([s, 1]) part, in place
template <class R>
__host__ __device__ inline void split5(R* b, R s, bool keep_left)
{
    R w[6], L[6], Rt[6];
    for (int i = 0; i < 6; ++i) w[i] = b[i];
    L[0] = w[0];
    Rt[5] = w[5];
    for (int r = 1; r < 6; ++r) {
        for (int i = 0; i < 6 - r; ++i) w[i] = w[i] + s * (w[i + 1] - w[i]);
        L[r] = w[0];
        Rt[5 - r] = w[5 - r];
    }
    for (int i = 0; i < 6; ++i) b[i] = keep_left ? L[i] : Rt[i];
}

// Bernstein coefficients of E on [t0, t1] from those on [0, 1] (Eq.
// subdivisionmatrix: the right part at t0, then the left part of that at
// (t1 - t0) / (1 - t0))
template <class R>
__host__ __device__ inline void restrict5(const R* b01, R t0, R t1, R* b)
{
    for (int i = 0; i < 6; ++i) b[i] = b01[i];
    if (t0 > R(0)) split5(b, t0, false);
    if (t1 < R(1)) split5(b, t0 < R(1) ? (t1 - t0) / (R(1) - t0) : R(1), true);
}

template <class R>
__host__ __device__ inline R horner5(const R* e, R u)
{
    return e[0] + u * (e[1] + u * (e[2] + u * (e[3] + u * (e[4] + u * e[5]))));
}

// sign changes of degree-5 Bernstein coefficients whose magnitude exceeds
// tol; `uncertain` is set when a coefficient within tol could change the
// count (at an end, between two certain coefficients of the same sign, or
// in a run of two or more)
template <class R>
__host__ __device__ inline int certain_changes5(const R* b, R tol, bool& uncertain)
{
    int v = 0, last = 0, run = 0;
    for (int i = 0; i < 6; ++i) {
        const int sg = b[i] > tol ? 1 : (b[i] < -tol ? -1 : 0);
        if (sg == 0) {
            if (i == 0 || i == 5) uncertain = true;
            ++run;
            continue;
        }
        if (run > 0 && (run > 1 || last == sg)) uncertain = true;
        run = 0;
        if (last != 0 && sg != last) ++v;
        last = sg;
    }
    return v;
}

struct ClipOut {
    int n_min;        // interior minima found (pieces where E goes from - to +)
    int rounds;       // clipping rounds run
    bool unsure;      // a decision rested on a value within its rounding bound
};

// Every local minimum of D on [0, 1] by the paper's search; returns the best
// minimiser.  Each piece is certified by the sign changes of E's Bernstein
// coefficients on it (an upper bound of its roots, of the same parity): at
// most one, none of them within tolE, after halving the piece up to three
// times; a part that stays uncertified (the closed-form roots of E', in the
// precision R, may have missed one) sets out.unsure.  second[0..2]: the second and third smallest D among the local
// minima and the minimiser of the second (as the sign-variation isolation
// reports them).  tolE: the rounding bound of E's values (a sign within it
// is not certain); rounds: clipping rounds per piece at most.
template <class R>
__host__ __device__ inline R clip_min(const R* c, R tolE, int rounds, R* second, ClipOut& out)
{
    R e[6], b01[6];
    power_E(c, e);
    // Bernstein form on [0, 1]: b = T e (Sec. 4.3, degree 5)
    b01[0] = e[0];
    b01[1] = e[0] + R(0.2) * e[1];
    b01[2] = e[0] + R(0.4) * e[1] + R(0.1) * e[2];
    b01[3] = e[0] + R(0.6) * e[1] + R(0.3) * e[2] + R(0.1) * e[3];
    b01[4] = e[0] + R(0.8) * e[1] + R(0.6) * e[2] + R(0.4) * e[3] + R(0.2) * e[4];
    b01[5] = e[0] + e[1] + e[2] + e[3] + e[4] + e[5];
    out.n_min = 0;
    out.rounds = 0;
    out.unsure = false;
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
    auto Dat = [&](R u) {
        R E, Ep;
        return eval_E(c, R(0), R(0), R(0), u, E, Ep);
    };
    // monotone decomposition: roots of E' = sum k e_k u^(k-1) in (0, 1)
    R cp[5] = { e[1], R(2) * e[2], R(3) * e[3], R(4) * e[4], R(5) * e[5] }, rt[4];
    const int nr = quartic_roots(cp, rt);
    R cut[6];
    int nc = 0;
    cut[nc++] = R(0);
    for (int i = 0; i < nr; ++i)
        if (rt[i] > R(0) && rt[i] < R(1)) cut[nc++] = rt[i];
    for (int i = 2; i < nc; ++i)  // sort the interior cuts
        for (int j = i; j > 1 && cut[j] < cut[j - 1]; --j) {
            const R t = cut[j];
            cut[j] = cut[j - 1];
            cut[j - 1] = t;
        }
    cut[nc++] = R(1);
    // the segment's ends (Property 2 for a segment: an end is a candidate
    // where D does not fall into the segment)
    const R E0 = horner5(e, R(0)), E1 = horner5(e, R(1));
    if (E0 >= -tolE) local_min(Dat(R(0)), R(0));
    if (E1 <= tolE) local_min(Dat(R(1)), R(1));
    // every piece, certified by the sign changes of E's Bernstein
    // coefficients on it (at most one, none of them within its rounding
    // bound), halved up to three times where the control polygon is not yet
    // close enough to E; Property 1 on each certified part
    struct Part {
        R b[6];
        R lo, hi;
        int depth;
    };
    for (int k = 0; k + 1 < nc; ++k) {
        if (!(cut[k + 1] > cut[k])) continue;
        Part st[5];
        int top = 0;
        restrict5(b01, cut[k], cut[k + 1], st[0].b);
        st[0].lo = cut[k];
        st[0].hi = cut[k + 1];
        st[0].depth = 0;
        top = 1;
        while (top > 0) {
            Part pt = st[--top];
            bool unc = false;
            const int v = certain_changes5(pt.b, tolE, unc);
            if (!unc && v >= 2 && pt.depth < 3) {
                const R mid = R(0.5) * (pt.lo + pt.hi);
                Part l = pt, r = pt;
                split5(l.b, R(0.5), true);
                split5(r.b, R(0.5), false);
                l.hi = mid;
                r.lo = mid;
                l.depth = r.depth = pt.depth + 1;
                st[top++] = r;
                st[top++] = l;
                continue;
            }
            if (unc || v >= 2) out.unsure = true;
            // Property 1: a minimum inside only where E goes from - to +
            if (!(pt.b[0] < R(0) && pt.b[5] > R(0))) continue;
            R b[6];
            for (int i = 0; i < 6; ++i) b[i] = pt.b[i];
            R lo = pt.lo, hi = pt.hi;
            const R wmin = R(1e-6) * (cut[k + 1] - cut[k]);
            for (int rd = 0; rd < rounds && hi - lo > wmin; ++rd) {
                // the convex hull of (i/5, b_i) cut with the axis: the
                // extreme crossings of the segments joining a negative and
                // a positive control point
                R zmin = R(1), zmax = R(0);
                for (int i = 0; i < 6; ++i)
                    for (int j = i + 1; j < 6; ++j)
                        if ((b[i] < R(0)) != (b[j] < R(0))) {
                            const R z = (R(i) + R(j - i) * b[i] / (b[i] - b[j])) * R(0.2);
                            zmin = fmin(zmin, z);
                            zmax = fmax(zmax, z);
                        }
                if (!(zmax > zmin)) break;
                if (zmax - zmin > R(0.5)) {
                    // bisect: the half whose end values differ in sign
                    R l[6];
                    for (int i = 0; i < 6; ++i) l[i] = b[i];
                    split5(l, R(0.5), true);
                    if ((l[0] < R(0)) != (l[5] < R(0))) {
                        for (int i = 0; i < 6; ++i) b[i] = l[i];
                        zmin = R(0);
                        zmax = R(0.5);
                    } else {
                        split5(b, R(0.5), false);
                        zmin = R(0.5);
                        zmax = R(1);
                    }
                } else {
                    split5(b, zmin, false);
                    split5(b, zmin < R(1) ? (zmax - zmin) / (R(1) - zmin) : R(1), true);
                }
                const R w = hi - lo;
                hi = lo + zmax * w;
                lo = lo + zmin * w;
                ++out.rounds;
            }
            // the root of the last clip's chord
            const R den = b[5] - b[0];
            R u = den != R(0) ? lo + (hi - lo) * (-b[0] / den) : R(0.5) * (lo + hi);
            u = fmin(fmax(u, lo), hi);
            local_min(Dat(u), u);
            ++out.n_min;
        }
    }
    if (second) {
        second[0] = m2;
        second[1] = m3;
        second[2] = u2;
    }
    return m1 < R(INFINITY) ? u1 : (Dat(R(1)) < Dat(R(0)) ? R(1) : R(0));
}

}  // namespace bspl
