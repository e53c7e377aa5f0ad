"""Pins of the oracle's rational-curve (NURBS) functions against facts fixed
by mathematics, none of them a retyping of the oracle's own formulas:

* evaluation against SciPy's B-spline evaluator (numerator / denominator of
  the homogeneous form), and on exact circles against |C - c| = r, the
  tangent condition (C - c).C' = 0 and its derivative (C - c).C'' = -|C'|^2;
* projection on circles against the closed-form distance to a circle, and on
  tiny random NURBS against brute force;
* the homogeneous span extraction against textbook knot insertion;
* the Hermite cubic against its interpolation conditions (finite
  differences of an explicit rational Bernstein sum);
* the certified bound against sampled deviations, and the decomposition's
  segments against the original curve at the tolerance;
* equal weights reduce every result to the non-rational one.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import oracle as O
from paper_2504_11498_gb300 import synth


def rbez(H, u):
    """Explicit rational Bernstein sum of homogeneous points H [p+1][4]."""
    H = np.asarray(H)
    p = H.shape[0] - 1
    u = np.atleast_1d(u)[:, None]
    S = sum(math.comb(p, i) * u ** i * (1 - u) ** (p - i) * H[i] for i in range(p + 1))
    return S[:, :3] / S[:, 3:]


def cubic(R, u):
    u = np.atleast_1d(u)[:, None]
    return sum(math.comb(3, i) * u ** i * (1 - u) ** (3 - i) * R[i] for i in range(4))


def random_rpiece(rng, p, wlo=0.2, whi=5.0):
    P = rng.uniform(-1, 1, size=(p + 1, 3))
    w = np.exp(rng.uniform(np.log(wlo), np.log(whi), size=p + 1))
    return np.concatenate([P * w[:, None], w[:, None]], axis=1)


def small_nurbs(seed=11, n=12, w_range=(0.5, 2.0)):
    cs, qs = synth.nurbs_curve_set(seed=seed, n_curves=n, n_proj=400, n_inv=0, ncp_range=(8, 14),
                                   w_range=w_range)
    return cs, qs


# ------------------------------------------------------------ evaluation

def test_eval_matches_scipy_homogeneous_ratio():
    cs, _ = small_nurbs()
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        w = cs.curve_weights(c)
        num = BSpline(U, P * w[:, None], p)
        den = BSpline(U, w, p)
        t = np.linspace(U[p], U[len(P)], 257)
        ref = num(t) / den(t)[:, None]
        got = O.eval_curves(cs, np.full(len(t), c, np.int32), t)[0]
        assert np.abs(got - ref).max() <= 1e-14, c


def test_circle_eval_radius_tangent_curvature():
    cs, _, centre, radius, normal = synth.nurbs_circles(n_curves=8, n_proj=1)
    t = np.linspace(0.0, 1.0, 1001)
    for c in range(cs.n):
        C, C1, C2 = O.eval_curves(cs, np.full(len(t), c, np.int32), t)
        d = C - centre[c]
        r = radius[c]
        assert np.abs(np.linalg.norm(d, axis=1) - r).max() <= 4e-15 * (1 + r)
        # in the circle's plane
        assert np.abs(d @ normal[c]).max() <= 4e-15
        # tangent: (C - c).C' = 0, and its derivative (C - c).C'' = -|C'|^2
        sp = np.linalg.norm(C1, axis=1)
        assert np.abs(np.einsum("ij,ij->i", d, C1)).max() <= 1e-13 * r * sp.max()
        assert np.allclose(np.einsum("ij,ij->i", d, C2), -sp ** 2, rtol=1e-12, atol=1e-12 * sp.max() ** 2)


def test_rational_derivatives_finite_differences():
    cs, _ = small_nurbs(seed=12)
    rng = np.random.default_rng(3)
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        a, b = U[p], U[len(P)]
        inner = np.unique(U[(U > a) & (U < b)])
        t = rng.uniform(a, b, size=40)
        # keep away from knots, where the derivatives of low-continuity curves jump
        if len(inner):
            t = t[np.min(np.abs(t[:, None] - inner[None, :]), axis=1) > 1e-3 * (b - a)]
        t = t[(t > a + 1e-3 * (b - a)) & (t < b - 1e-3 * (b - a))]
        h = 1e-6 * (b - a)
        idx = np.full(len(t), c, np.int32)
        C, C1, C2 = O.eval_curves(cs, idx, t)
        Cp, C1p, _ = O.eval_curves(cs, idx, t + h)
        Cm, C1m, _ = O.eval_curves(cs, idx, t - h)
        sc1 = np.abs(C1).max() + 1e-300
        sc2 = np.abs(C2).max() + 1e-300
        assert np.abs((Cp - Cm) / (2 * h) - C1).max() <= 1e-6 * max(sc1, sc2 * (b - a)), c
        assert np.abs((C1p - C1m) / (2 * h) - C2).max() <= 1e-5 * sc2 + 1e-6 * sc1 / (b - a), c


def test_equal_weights_reduce_to_non_rational():
    cs, qs = synth.curve_set(seed=9, n_curves=10, n_proj=300, n_inv=0, ncp_range=(8, 16))
    rat = synth.CurveSet(cs.degree, cs.knot_off, cs.knots, cs.cp_off, cs.cps, np.full(len(cs.cps), 2.5))
    t = np.random.default_rng(0).uniform(0, 1, 500)
    qc = np.random.default_rng(1).integers(0, cs.n, 500).astype(np.int32)
    for a, b in zip(O.eval_curves(cs, qc, t), O.eval_curves(rat, qc, t)):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-13)
    # the decomposition takes the non-rational route: identical arrays
    d0, d1 = O.decompose_curves(cs, 1e-9), O.decompose_curves(rat, 1e-9)
    assert np.array_equal(d0.seg_off, d1.seg_off)
    assert np.array_equal(d0.ctrl, d1.ctrl) and np.array_equal(d0.prange, d1.prange)
    _, dd0 = O.project_curves(cs, qs.proj_curve, qs.proj_xyz)
    _, dd1 = O.project_curves(rat, qs.proj_curve, qs.proj_xyz)
    assert np.allclose(dd0, dd1, rtol=1e-12, atol=1e-14)


def test_invalid_weights_rejected():
    cs, _ = small_nurbs(n=3)
    for bad in (0.0, -1.0, np.nan, np.inf):
        w = cs.weights.copy()
        w[5] = bad
        with pytest.raises(ValueError):
            O.decompose_curves(synth.CurveSet(cs.degree, cs.knot_off, cs.knots, cs.cp_off, cs.cps, w), 1e-6)


# ------------------------------------------------- homogeneous decomposition

def test_homogeneous_span_bezier_matches_knot_insertion():
    cs, _ = small_nurbs(seed=13)
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        w = cs.curve_weights(c)
        H = O.rspan_bezier(p, U, P, w)
        num = O.boehm_bezier(p, U, P * w[:, None])
        den = O.boehm_bezier(p, U, np.stack([w, np.zeros_like(w), np.zeros_like(w)], 1))
        assert H.shape[0] == num.shape[0]
        assert np.abs(H[:, :, :3] - num).max() <= 1e-13 * (1 + np.abs(num).max())
        assert np.abs(H[:, :, 3] - den[:, :, 0]).max() <= 1e-13 * w.max()
        assert np.all(H[:, :, 3] > 0)


def test_hermite_interpolates_ends_and_tangents():
    rng = np.random.default_rng(21)
    for p in range(1, 9):
        for _ in range(10):
            H = random_rpiece(rng, p)
            R = O.rhermite(H)
            assert np.allclose(R[0], rbez(H, 0.0)[0], atol=1e-14)
            assert np.allclose(R[3], rbez(H, 1.0)[0], atol=1e-14)
            h = 1e-6
            d0 = (rbez(H, h)[0] - rbez(H, 0.0)[0]) / h           # one-sided at the ends
            d1 = (rbez(H, 1.0)[0] - rbez(H, 1.0 - h)[0]) / h
            d0c = (-3 * rbez(H, 0.0)[0] + 4 * rbez(H, h)[0] - rbez(H, 2 * h)[0]) / (2 * h)
            d1c = (3 * rbez(H, 1.0)[0] - 4 * rbez(H, 1.0 - h)[0] + rbez(H, 1.0 - 2 * h)[0]) / (2 * h)
            sc = 1 + np.abs(d0).max() + np.abs(d1).max()
            assert np.abs(3 * (R[1] - R[0]) - d0c).max() <= 1e-6 * sc, (p, R, d0c)
            assert np.abs(3 * (R[3] - R[2]) - d1c).max() <= 1e-6 * sc, (p, R, d1c)


def test_bound_covers_sampled_deviation_and_is_not_loose():
    rng = np.random.default_rng(22)
    u = np.linspace(0.0, 1.0, 2001)
    ratios = []
    for p in range(1, 9):
        for _ in range(25):
            H = random_rpiece(rng, p)
            R = O.rhermite(H)
            b2 = O.rbound2(H, R)
            dev = np.linalg.norm(rbez(H, u) - cubic(R, u), axis=1).max()
            assert dev ** 2 <= b2 * (1 + 1e-9) + 1e-28, (p, dev, math.sqrt(b2))
            if dev > 1e-6:
                ratios.append(math.sqrt(b2) / dev)
    # the bound is within a modest factor of the true deviation
    assert np.median(ratios) < 20.0 and max(ratios) < 400.0, (np.median(ratios), max(ratios))


def test_bound_vanishes_on_polynomial_cubics():
    rng = np.random.default_rng(23)
    for p in (1, 2, 3):
        P = rng.uniform(-1, 1, size=(p + 1, 3))
        H = np.concatenate([3.0 * P, np.full((p + 1, 1), 3.0)], axis=1)
        R = O.rhermite(H)
        assert O.rbound2(H, R) <= 1e-28
        u = np.linspace(0, 1, 11)
        assert np.abs(cubic(R, u) - rbez(H, u)).max() <= 1e-14


def test_rhalve_reparameterises():
    rng = np.random.default_rng(24)
    u = np.linspace(0.0, 1.0, 33)
    for p in range(1, 9):
        H = random_rpiece(rng, p)
        L, R = O.rhalve(H)
        assert np.abs(rbez(L, u) - rbez(H, 0.5 * u)).max() <= 1e-13
        assert np.abs(rbez(R, u) - rbez(H, 0.5 + 0.5 * u)).max() <= 1e-13


@pytest.mark.parametrize("tol", [1e-4, 1e-7])
def test_decomposition_segments_within_tolerance(tol):
    cs, _ = small_nurbs(seed=14, n=10)
    dec = O.decompose_curves(cs, tol)
    assert dec.status == 0
    diag = O.curve_diag(cs)
    u = np.linspace(0.0, 1.0, 65)
    worst = 0.0
    for c in range(cs.n):
        for s in range(dec.seg_off[c], dec.seg_off[c + 1]):
            t0, t1 = dec.prange[s]
            t = t0 + u * (t1 - t0)
            C = O.eval_curves(cs, np.full(len(t), c, np.int32), t)[0]
            dev = np.linalg.norm(C - cubic(dec.ctrl[s], u), axis=1).max()
            worst = max(worst, dev / (tol * diag[c]))
        # segments tile the domain in order
        p, U, P = cs.curve(c)
        pr = dec.prange[dec.seg_off[c]:dec.seg_off[c + 1]]
        assert pr[0, 0] == U[p] and pr[-1, 1] == U[len(P)]
        assert np.all(pr[1:, 0] == pr[:-1, 1])
    assert worst <= 1.0 + 1e-9, worst


def test_circle_segment_count_scales_with_fourth_root():
    cs, _, _, _, _ = synth.nurbs_circles(n_curves=4, n_proj=1)
    n6 = O.decompose_curves(cs, 1e-6).total
    n10 = O.decompose_curves(cs, 1e-10).total
    # Hermite cubics: error ~ h^4, so 1e4 times tighter needs ~10x the pieces
    assert 4 <= n10 / n6 <= 20, (n6, n10)


# ------------------------------------------------------------- projection

def test_derivative_bounds_cover_samples():
    """The projection's branch and bound rests on bounds of |C'| and |C''|
    per span; sampled derivatives never exceed them."""
    cs, _ = small_nurbs(seed=16, n=10, w_range=(0.25, 4.0))
    u = np.linspace(0.0, 1.0, 201)[1:-1]
    ratios = []
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        w = cs.curve_weights(c)
        for q in range(p, len(P)):
            if not U[q] < U[q + 1]:
                continue
            V, A = O.curve_deriv_bounds(p, U, P, w, q)
            t = U[q] + u * (U[q + 1] - U[q])
            _, C1, C2 = O.eval_curves(cs, np.full(len(t), c, np.int32), t)
            v, a = np.linalg.norm(C1, axis=1).max(), np.linalg.norm(C2, axis=1).max()
            assert v <= V * (1 + 1e-12) and a <= A * (1 + 1e-12), (c, q, v, V, a, A)
            ratios.append(V / v)
    assert np.median(ratios) < 10.0, np.median(ratios)


def test_circle_projection_closed_form():
    cs, qs, centre, radius, normal = synth.nurbs_circles(n_curves=16, n_proj=3000)
    t, d = O.project_curves(cs, qs.proj_curve, qs.proj_xyz)
    c = qs.proj_curve
    v = qs.proj_xyz - centre[c]
    h = np.einsum("ij,ij->i", v, normal[c])
    inplane = v - h[:, None] * normal[c]
    rho = np.linalg.norm(inplane, axis=1)
    exact = np.sqrt(h * h + (rho - radius[c]) ** 2)
    assert np.abs(d - exact).max() <= 1e-13
    # the foot point is c + r (in-plane direction) away from the axis
    ok = rho > 1e-3 * radius[c]
    foot = O.eval_curves(cs, c, t)[0]
    ref = centre[c] + radius[c, None] * inplane / np.maximum(rho, 1e-300)[:, None]
    assert np.abs(foot[ok] - ref[ok]).max() <= 1e-6 * radius.max()


def test_projection_brute_force_tiny():
    cs, qs = small_nurbs(seed=15, n=6, w_range=(0.25, 4.0))
    qc, q = qs.proj_curve[:120], qs.proj_xyz[:120]
    t, d = O.project_curves(cs, qc, q)
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        tt = np.linspace(U[p], U[len(P)], 200_001)
        S = O.eval_curves(cs, np.full(len(tt), c, np.int32), tt)[0]
        sel = np.where(qc == c)[0]
        for k in sel:
            brute = np.sqrt(((S - q[k]) ** 2).sum(1)).min()
            assert d[k] <= brute + 1e-15
            assert brute - d[k] <= 1e-7, (c, k, brute, d[k])
        # the returned parameter reproduces the distance
        Ck = O.eval_curves(cs, qc[sel], t[sel])[0]
        assert np.allclose(np.linalg.norm(Ck - q[sel], axis=1), d[sel], rtol=0, atol=1e-14)


def test_edge_set_projection_brute_force_and_quarter_circle():
    """Rational edge cases (a line with unequal weights, a quarter circle, a
    C0 joint, one degree-7 span, the domain [-3, 5], weights over 50:1):
    the oracle's projection against brute force, the quarter circle against
    its closed form, the decomposition within the tolerance."""
    cs = synth.nurbs_edge_set()
    rng = np.random.default_rng(8)
    lo, hi = synth.cp_boxes(cs)
    qc = np.repeat(np.arange(cs.n, dtype=np.int32), 40)
    q = synth._box_queries(rng, lo, hi, qc, scale=1.5)
    t, d = O.project_curves(cs, qc, q)
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        tt = np.linspace(U[p], U[len(P)], 200_001)
        S = O.eval_curves(cs, np.full(len(tt), c, np.int32), tt)[0]
        for k in np.where(qc == c)[0]:
            brute = np.sqrt(((S - q[k]) ** 2).sum(1)).min()
            assert d[k] <= brute + 1e-15 and brute - d[k] <= 1e-7, (c, k, brute, d[k])
    # quarter circle of radius 1 about the origin in z = 0
    k = np.where(qc == 1)[0]
    v = q[k]
    rho = np.linalg.norm(v[:, :2], axis=1)
    ang = np.arctan2(v[:, 1], v[:, 0])
    on_arc = (ang >= 0) & (ang <= np.pi / 2)
    exact = np.where(on_arc, np.sqrt(v[:, 2] ** 2 + (rho - 1) ** 2),
                     np.minimum(np.linalg.norm(v - [1, 0, 0], axis=1), np.linalg.norm(v - [0, 1, 0], axis=1)))
    assert np.abs(d[k] - exact).max() <= 1e-13
    dec = O.decompose_curves(cs, 1e-8)
    assert dec.status == 0
    u = np.linspace(0.0, 1.0, 33)
    diag = O.curve_diag(cs)
    for c in range(cs.n):
        for s in range(dec.seg_off[c], dec.seg_off[c + 1]):
            t0, t1 = dec.prange[s]
            C = O.eval_curves(cs, np.full(len(u), c, np.int32), t0 + u * (t1 - t0))[0]
            assert np.linalg.norm(C - cubic(dec.ctrl[s], u), axis=1).max() <= 1e-8 * diag[c] * (1 + 1e-9)
