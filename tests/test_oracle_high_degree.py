"""Pins of the oracle for curves of high degree (up to 63; the paper stops
at 31).  The decomposition extracts each span by the power-basis matrix
route up to degree 7 and from the blossom above, because the matrix route's
FP64 error grows about tenfold every two degrees:

* the blossom extraction against textbook knot insertion at degrees 33..63;
* the matrix route's loss of digits at high degree (why the switch), and
  the blossom's exactness there;
* evaluation against SciPy's B-spline evaluator at degree 50;
* the decomposition's segments within the tolerance of the original curve;
* projection against brute force on a degree-45 curve.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import oracle as O
from paper_2504_11498_gb300 import synth


def high_curve(rng, p, ncp, repeat_prob=0.1):
    U = synth.random_clamped_knots(rng, p, ncp, repeat_prob)
    return U, rng.uniform(0.0, 1.0, size=(ncp, 3))


@pytest.mark.parametrize("p", [33, 40, 50, 63])
def test_blossom_extraction_matches_knot_insertion(p):
    rng = np.random.default_rng(p)
    U, P = high_curve(rng, p, p + 6)
    Qb = O.span_blossom(p, U, P)
    Qk = O.boehm_bezier(p, U, P)
    assert Qb.shape == Qk.shape and Qb.shape[0] >= 1
    assert np.abs(Qb - Qk).max() <= 1e-12


def test_matrix_route_error_by_degree():
    """Against knot insertion: the matrix route stays within 1e-13 up to
    degree 7 and passes 1e-11 by degree 15 and 1e-4 by degree 31; the blossom
    stays within 1e-14 at every degree (hence the switch above 7)."""
    rng = np.random.default_rng(1)
    err_m, err_b = {}, {}
    for p in (3, 5, 7, 15, 31):
        em = eb = 0.0
        for _ in range(20):
            U, P = high_curve(rng, p, p + int(rng.integers(1, 12)))
            Qk = O.boehm_bezier(p, U, P)
            em = max(em, np.abs(O.span_bezier(p, U, P) - Qk).max())
            eb = max(eb, np.abs(O.span_blossom(p, U, P) - Qk).max())
        err_m[p], err_b[p] = em, eb
    assert max(err_m[3], err_m[5], err_m[7]) <= 1e-13, err_m
    assert err_m[15] >= 1e-11 and err_m[31] >= 1e-4, err_m
    assert max(err_b.values()) <= 1e-14, err_b


def test_matrix_route_loses_digits_at_high_degree():
    """At degree 40 the power-basis route is off by orders of magnitude more
    than the tolerances in use, the blossom is not (this is the reason the
    extraction switches above degree 31)."""
    rng = np.random.default_rng(4)
    U, P = high_curve(rng, 40, 46, repeat_prob=0.0)
    Qk = O.boehm_bezier(40, U, P)
    err_matrix = np.abs(O.span_bezier(40, U, P) - Qk).max()
    err_blossom = np.abs(O.span_blossom(40, U, P) - Qk).max()
    assert err_blossom <= 1e-13 < 1e-8 <= err_matrix, (err_blossom, err_matrix)
    # at low degree both routes agree
    U, P = high_curve(rng, 5, 12)
    assert np.abs(O.span_bezier(5, U, P) - O.span_blossom(5, U, P)).max() <= 1e-14


def test_high_degree_eval_matches_scipy():
    rng = np.random.default_rng(5)
    U, P = high_curve(rng, 50, 60)
    cs = synth.pack_curves([50], [U], [P])
    t = np.linspace(0, 1, 301)
    C, C1, C2 = O.eval_curves(cs, np.zeros(len(t), np.int32), t)
    S = BSpline(U, P, 50)
    assert np.abs(C - S(t)).max() <= 1e-13
    assert np.abs(C1 - S.derivative(1)(t)).max() <= 1e-9 * np.abs(C1).max()


@pytest.mark.parametrize("p,tol", [(40, 1e-8), (63, 1e-6)])
def test_high_degree_decomposition_within_tolerance(p, tol):
    rng = np.random.default_rng(10 + p)
    U, P = high_curve(rng, p, p + 5)
    cs = synth.pack_curves([p], [U], [P])
    dec = O.decompose_curves(cs, tol)
    assert dec.status == 0 and dec.total >= 1
    diag = O.curve_diag(cs)[0]
    u = np.linspace(0.0, 1.0, 65)
    worst = 0.0
    for s in range(dec.total):
        t0, t1 = dec.prange[s]
        C = O.eval_curves(cs, np.zeros(len(u), np.int32), t0 + u * (t1 - t0))[0]
        R = dec.ctrl[s]
        B = sum(math.comb(3, i) * u[:, None] ** i * (1 - u[:, None]) ** (3 - i) * R[i] for i in range(4))
        worst = max(worst, np.linalg.norm(C - B, axis=1).max() / (tol * diag))
    assert worst <= 1.0 + 1e-9, worst
    pr = dec.prange
    assert pr[0, 0] == U[p] and pr[-1, 1] == U[len(P)] and np.all(pr[1:, 0] == pr[:-1, 1])


def test_high_degree_projection_brute_force():
    rng = np.random.default_rng(6)
    U, P = high_curve(rng, 45, 52)
    cs = synth.pack_curves([45], [U], [P])
    lo, hi = synth.cp_boxes(cs)
    qc = np.zeros(60, np.int32)
    q = synth._box_queries(rng, lo, hi, qc, scale=1.4)
    t, d = O.project_curves(cs, qc, q)
    tt = np.linspace(0.0, 1.0, 200_001)
    S = O.eval_curves(cs, np.zeros(len(tt), np.int32), tt)[0]
    for k in range(len(qc)):
        brute = np.sqrt(((S - q[k]) ** 2).sum(1)).min()
        assert d[k] <= brute + 1e-15 and brute - d[k] <= 1e-7, (k, brute, d[k])
