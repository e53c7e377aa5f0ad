"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself:
SciPy's independent B-spline evaluator, closed forms, exact polynomial roots,
Gauss-Legendre quadrature, the matrices printed in the paper (tests/golden/),
brute force on tiny inputs, and invariants such as partition of unity.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline
from scipy.optimize import minimize, minimize_scalar

from oracle import oracle as O
from paper_2504_11498_gb300 import synth

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers

def bez(Q, u):
    """Explicit Bernstein sum of a Bezier curve, Q [p+1][3], u [k] -> [k][3]."""
    Q = np.asarray(Q)
    p = Q.shape[0] - 1
    u = np.atleast_1d(u)[:, None]
    return sum(math.comb(p, i) * u ** i * (1 - u) ** (p - i) * Q[i] for i in range(p + 1))


def bez_patch(Q, u, v):
    """Explicit tensor Bernstein sum, Q [m+1][n+1][3]."""
    m, n = Q.shape[0] - 1, Q.shape[1] - 1
    Bu = np.array([math.comb(m, i) * u ** i * (1 - u) ** (m - i) for i in range(m + 1)])
    Bv = np.array([math.comb(n, j) * v ** j * (1 - v) ** (n - j) for j in range(n + 1)])
    return np.einsum("i,j,ijc->c", Bu, Bv, Q)


def scipy_curve(p, U, P):
    return BSpline(np.asarray(U), np.asarray(P), p)


def scipy_surface(pu, pv, U, V, P, u, v, du=0, dv=0):
    bu = BSpline(U, np.eye(P.shape[0]), pu)
    bv = BSpline(V, np.eye(P.shape[1]), pv)
    Nu = (bu.derivative(du) if du else bu)(u)
    Nv = (bv.derivative(dv) if dv else bv)(v)
    return np.einsum("i,j,ijc->c", Nu, Nv, P)


def rand_curve(rng, p, ncp, repeat=0.1):
    return synth.random_clamped_knots(rng, p, ncp, repeat), rng.uniform(0, 1, (ncp, 3))


def greville(U, p, n):
    return np.array([np.mean(U[i + 1:i + p + 1]) for i in range(n)])


def diag_of(P):
    P = np.asarray(P).reshape(-1, 3)
    return float(np.linalg.norm(P.max(0) - P.min(0)))


# ----------------------------------------------------- evaluation (Sec. 3)

@pytest.mark.parametrize("p", range(1, 8))
def test_partition_of_unity_and_support(p):
    rng = np.random.default_rng(100 + p)
    U, _ = rand_curve(rng, p, 24)
    for t in rng.uniform(0, 1, 1500):
        s, N = O.basis(p, U, t)
        assert abs(N.sum() - 1.0) <= 4e-15
        assert (N >= -1e-17).all()
        assert U[s] <= t <= U[s + 1] and U[s] < U[s + 1]


@pytest.mark.parametrize("p", range(1, 8))
def test_eval_matches_scipy(p):
    rng = np.random.default_rng(200 + p)
    U, P = rand_curve(rng, p, 30, repeat=0.0)
    cs = synth.pack_curves([p], [U], [P])
    t = rng.uniform(0, 1, 400)
    C, C1, C2 = O.eval_curves(cs, np.zeros(len(t), np.int32), t)
    sp = scipy_curve(p, U, P)
    scale = 1.0 + np.abs(sp(t)).max()
    assert np.abs(C - sp(t)).max() <= 1e-13 * scale
    d1 = sp.derivative(1)(t)
    assert np.abs(C1 - d1).max() <= 1e-11 * (1 + np.abs(d1).max())
    if p >= 2:
        d2 = sp.derivative(2)(t)
        assert np.abs(C2 - d2).max() <= 1e-10 * (1 + np.abs(d2).max())


def test_degree1_is_polyline():
    rng = np.random.default_rng(7)
    U, P = rand_curve(rng, 1, 9, repeat=0.0)
    cs = synth.pack_curves([1], [U], [P])
    t = rng.uniform(0, 1, 300)
    C, _, _ = O.eval_curves(cs, np.zeros(len(t), np.int32), t)
    for k, tk in enumerate(t):
        i = np.searchsorted(U, tk, side="right") - 1  # U[i] <= t < U[i+1]
        a = (tk - U[i]) / (U[i + 1] - U[i])
        ref = P[i - 1] + a * (P[i] - P[i - 1])
        assert np.abs(C[k] - ref).max() <= 1e-15 * 4


# ------------------------------------------- decomposition (Sec. 4.2.1)

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_bezier_extraction_reproduces_curve(p):
    rng = np.random.default_rng(300 + p)
    U, P = rand_curve(rng, p, 20, repeat=0.2)
    Qb = O.boehm_bezier(p, U, P)
    Qm = O.span_bezier(p, U, P)
    spans = [q for q in range(p, len(P)) if U[q] < U[q + 1]]
    assert len(spans) == Qb.shape[0] == Qm.shape[0]
    sp = scipy_curve(p, U, P)
    d = diag_of(P)
    for k, q in enumerate(spans):
        u = rng.uniform(0, 1, 50)
        t = U[q] + u * (U[q + 1] - U[q])
        ref = sp(t)
        assert np.abs(bez(Qb[k], u) - ref).max() <= 1e-14 * 16 * d
        assert np.abs(bez(Qm[k], u) - ref).max() <= 1e-14 * 16 * d
    # the two routes agree with each other at rounding level
    assert np.abs(Qb - Qm).max() <= 1e-13 * d


def test_paper_global_matrices_match_local_route():
    """Q = B_p^{-1} M_{q,p,T} A_{q,p,T} P with the p+1 control points
    P_{q-p..q} (Eqs. bsplinematrix, Mqpt, decomfinal; B_p^{-1} = T), evaluated
    exactly in rationals, equals the local-u route to rounding.  Evaluated in
    FP64 the global-t product loses digits (powers of t_q), which is why the
    method forms the product directly in u."""
    rng = np.random.default_rng(11)
    fp64_err = 0.0
    for p in (2, 3, 4, 5):
        U, P = rand_curve(rng, p, 10, repeat=0.0)
        Qm = O.span_bezier(p, U, P)
        spans = [q for q in range(p, len(P)) if U[q] < U[q + 1]]
        for k, q in enumerate(spans):
            Qx = O.tables.decomfinal_exact(U, q, p, P)
            assert np.abs(Qx - Qm[k]).max() <= 1e-14 * diag_of(P)
            Qf = O.tables.T(p) @ (O.tables.M_qpT(U[q], U[q + 1], p) @ O.tables.A_qpT(U, q, p)) @ P[q - p:q + 1]
            fp64_err = max(fp64_err, np.abs(Qf - Qx).max())
    assert fp64_err > 1e-13  # the global-t route is visibly worse in FP64


def test_elevation_exact():
    rng = np.random.default_rng(12)
    for n in (1, 2, 3, 5):
        Q = rng.uniform(0, 1, (n + 1, 3))
        E = O.elevate(Q)
        u = np.linspace(0, 1, 101)
        assert np.abs(bez(E, u) - bez(Q, u)).max() <= 1e-15 * 8


# ------------------------------------------ printed tables (Sec. 4.2.2, 4.3)

def _read_golden_matrix(name):
    rows = []
    for line in open(f"{GOLDEN}/{name}"):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line)
    return rows


def test_power_to_bernstein_T_matches_print():
    printed = np.array([[float(x) for x in r.split()] for r in _read_golden_matrix("power_to_bernstein_T5.txt")])
    assert np.allclose(O.tables.T(5), printed, rtol=0, atol=1e-15)
    # and it is the inverse of the Bernstein-to-power matrix
    assert np.allclose(O.tables.T(5) @ O.tables.bernstein_to_power(5), np.eye(6), atol=1e-13)


def test_subdivision_matrix_matches_print_and_halving():
    rows = _read_golden_matrix("subdivision_matrix_S.txt")
    for z in (0.5, 0.1, 0.37, 0.9):
        printed = np.array([[eval(e, {"z": z}) for e in r.split(";")] for r in rows])
        assert np.allclose(O.tables.S(z), printed, atol=1e-15)
    rng = np.random.default_rng(13)
    Q = rng.uniform(0, 1, (4, 3))
    L, R = O.halve(Q)
    S = O.tables.S(0.5)
    assert np.abs(L - S[:4] @ Q).max() <= 1e-15 * 4
    assert np.abs(R - S[4:] @ Q).max() <= 1e-15 * 4
    # S_L(z) Q traced at u is Q traced at z u (the left piece)
    z = 0.37
    u = np.linspace(0, 1, 21)
    assert np.abs(bez(O.tables.S(z)[:4] @ Q, u) - bez(Q, z * u)).max() <= 1e-14
    assert np.abs(bez(O.tables.S(z)[4:] @ Q, u) - bez(Q, z + (1 - z) * u)).max() <= 1e-14


@pytest.mark.parametrize("m,n", [(3, 3), (3, 4), (3, 7), (5, 5)])
def test_gram_matches_quadrature(m, n):
    x, w = np.polynomial.legendre.leggauss(16)
    t = 0.5 * (x + 1)
    w = 0.5 * w
    Bm = np.array([math.comb(m, i) * t ** i * (1 - t) ** (m - i) for i in range(m + 1)])
    Bn = np.array([math.comb(n, j) * t ** j * (1 - t) ** (n - j) for j in range(n + 1)])
    G = (Bm * w) @ Bn.T
    assert np.abs(G - O.tables.gram(m, n)).max() <= 1e-15 * 4
    for i in range(m + 1):
        for j in range(n + 1):
            assert abs(O.lib().orc_gram(m, n, i, j) - G[i, j]) <= 1e-15 * 4


# ----------------------------------------------- G1 reduction (Sec. 4.2.2)

def _eps(Q, d0, d1):
    """L2 error of Eq. epsl by 16-point Gauss-Legendre (exact for degree <= 31)."""
    p = Q.shape[0] - 1
    a = p / 3.0
    R = np.array([Q[0], Q[0] + a * d0 * (Q[1] - Q[0]), Q[p] - a * d1 * (Q[p] - Q[p - 1]), Q[p]])
    x, w = np.polynomial.legendre.leggauss(16)
    t = 0.5 * (x + 1)
    diff = bez(Q, t) - bez(R, t)
    return float(0.5 * np.sum(w * np.sum(diff * diff, axis=1)))


@pytest.mark.parametrize("p", [4, 5, 6, 7, 9])
def test_g1_reduction_is_stationary_point_of_eps(p):
    rng = np.random.default_rng(400 + p)
    for _ in range(20):
        Q = np.cumsum(rng.uniform(-0.3, 0.6, (p + 1, 3)), axis=0)
        R, d0, d1, regular = O.reduce_g1(Q)
        if not regular:
            continue
        h = 1e-4
        g0 = (_eps(Q, d0 + h, d1) - _eps(Q, d0 - h, d1)) / (2 * h)
        g1 = (_eps(Q, d0, d1 + h) - _eps(Q, d0, d1 - h)) / (2 * h)
        h00 = (_eps(Q, d0 + h, d1) - 2 * _eps(Q, d0, d1) + _eps(Q, d0 - h, d1)) / h ** 2
        h11 = (_eps(Q, d0, d1 + h) - 2 * _eps(Q, d0, d1) + _eps(Q, d0, d1 - h)) / h ** 2
        # a step of g/h would move delta by less than 1e-7 -> stationary
        assert abs(g0) <= 1e-7 * abs(h00) + 1e-13
        assert abs(g1) <= 1e-7 * abs(h11) + 1e-13
        # G1 end conditions (Eq. G1-condition)
        assert np.allclose(R[0], Q[0]) and np.allclose(R[3], Q[p])
        assert np.allclose(R[1] - R[0], (p / 3) * d0 * (Q[1] - Q[0]), atol=1e-14)
        assert np.allclose(R[3] - R[2], (p / 3) * d1 * (Q[p] - Q[p - 1]), atol=1e-14)


def test_printed_sign_breaks_optimality():
    """The appendix prints + before the delta1 terms; with that sign the
    solution is not a stationary point of eps (the method uses the sign
    derived from eps)."""
    rng = np.random.default_rng(41)
    worse = 0
    for _ in range(20):
        Q = np.cumsum(rng.uniform(-0.3, 0.6, (6, 3)), axis=0)
        R0, a0, b0, r0 = O.reduce_g1(Q, variant=0)
        R1, a1, b1, r1 = O.reduce_g1(Q, variant=1)
        if r0 and r1:
            worse += _eps(Q, a1, b1) > _eps(Q, a0, b0) * (1 + 1e-9)
    assert worse >= 15


@pytest.mark.parametrize("p", [4, 5, 7])
def test_reduction_of_elevated_cubic_is_exact(p):
    rng = np.random.default_rng(500 + p)
    C3 = rng.uniform(0, 1, (4, 3))
    Q = C3
    for _ in range(p - 3):
        Q = O.elevate(Q)
    R, d0, d1, regular = O.reduce_g1(Q)
    assert regular
    assert np.abs(R - C3).max() <= 1e-14
    assert abs(d0 - 1) <= 1e-12 and abs(d1 - 1) <= 1e-12


@pytest.mark.parametrize("p", [4, 5, 6, 7])
def test_certified_bound_dominates_sampled_deviation(p):
    rng = np.random.default_rng(600 + p)
    u = np.linspace(0, 1, 10001)
    for _ in range(10):
        Q = rng.uniform(0, 1, (p + 1, 3))
        R = O.to_cubic(Q)
        dev2 = np.max(np.sum((bez(Q, u) - bez(R, u)) ** 2, axis=1))
        assert O.bound2(Q, R) >= dev2 * (1 - 1e-12)


# -------------------------------------- error-controlled decomposition

def test_single_cubic_decomposes_exactly_into_13():
    cs, _ = synth.single_cubic(n_proj=10, n_inv=10)
    d = O.decompose_curves(cs, 0.0)
    assert list(d.seg_off) == [0, 13] and d.maxdepth == 0
    p, U, P = cs.curve(0)
    assert np.array_equal(d.ctrl, O.span_bezier(p, U, P))


@pytest.mark.parametrize("tol", [1e-4, 1e-7, 1e-10])
def test_decomposition_meets_tolerance(tol):
    rng = np.random.default_rng(31)
    degs, knots, cps = [], [], []
    for p in (2, 3, 4, 5, 6, 7):
        U, P = rand_curve(rng, p, 12, repeat=0.3)
        degs.append(p); knots.append(U); cps.append(P)
    cs = synth.pack_curves(degs, knots, cps)
    d = O.decompose_curves(cs, tol)
    assert d.status == O.OK
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        segs = range(d.seg_off[c], d.seg_off[c + 1])
        pr = d.prange[segs.start:segs.stop]
        # the pieces tile [t_p, t_{m+1}] in order
        assert pr[0, 0] == U[p] and pr[-1, 1] == U[len(P)]
        assert np.all(pr[1:, 0] == pr[:-1, 1]) and np.all(pr[:, 1] > pr[:, 0])
        if p <= 3:
            assert len(segs) == sum(U[q] < U[q + 1] for q in range(p, len(P)))
        sp = scipy_curve(p, U, P)
        thr = tol * diag_of(P)
        for k in segs:
            t0, t1 = d.prange[k]
            u = np.linspace(0, 1, 33)
            err = np.abs(bez(d.ctrl[k], u) - sp(t0 + u * (t1 - t0)))
            assert np.sqrt((err ** 2).sum(1)).max() <= thr + 1e-14 * 32


def test_decompose_rejects_bad_knots():
    U = np.array([0, 0, 0, 0.5, 0.4, 1, 1, 1.0])
    cs = synth.pack_curves([2], [U], [np.zeros((5, 3))])
    with pytest.raises(ValueError):
        O.decompose_curves(cs, 1e-6)


# ------------------------------------------------ projection (Sec. 3)

def test_projection_onto_line_closed_form():
    """A degree-5 B-spline with Greville control points is the straight
    segment a + t (b - a) (linear precision): t* = clamp((q-a).(b-a)/|b-a|^2)."""
    rng = np.random.default_rng(21)
    p, ncp = 5, 14
    U = synth.random_clamped_knots(rng, p, ncp, 0.0)
    a, b = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    P = a + greville(U, p, ncp)[:, None] * (b - a)
    cs = synth.pack_curves([p], [U], [P])
    q = rng.uniform(-1.5, 1.5, (300, 3))
    t, d = O.project_curves(cs, np.zeros(len(q), np.int32), q)
    tr = np.clip((q - a) @ (b - a) / np.dot(b - a, b - a), 0, 1)
    dr = np.linalg.norm(q - (a + tr[:, None] * (b - a)), axis=1)
    assert np.abs(d - dr).max() <= 1e-13 * diag_of(P)
    # the minimiser's parameter is fixed only to ~sqrt(machine eps) by distances
    assert np.abs(t - tr).max() <= 1e-7


@pytest.mark.parametrize("elev", [0, 3])
def test_projection_onto_parabola_closed_form(elev):
    """Degree-2 Bezier (optionally elevated to degree 5): E(t) is a cubic whose
    real roots in [0,1], with the ends, contain the minimiser."""
    rng = np.random.default_rng(22 + elev)
    for _ in range(5):
        Q = rng.uniform(0, 1, (3, 3))
        Qe = Q
        for _ in range(elev):
            Qe = O.elevate(Qe)
        p = Qe.shape[0] - 1
        U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])
        cs = synth.pack_curves([p], [U], [Qe])
        a, b, c = Q[0], 2 * (Q[1] - Q[0]), Q[0] - 2 * Q[1] + Q[2]
        qs = rng.uniform(-0.5, 1.5, (60, 3))
        t, d = O.project_curves(cs, np.zeros(len(qs), np.int32), qs)
        for k, q in enumerate(qs):
            w = a - q
            coeffs = [2 * c @ c, 3 * b @ c, b @ b + 2 * w @ c, w @ b]
            cand = [0.0, 1.0] + [r.real for r in np.roots(coeffs) if abs(r.imag) < 1e-9 and 0 <= r.real <= 1]
            dist = [np.linalg.norm(a + b * s + c * s * s - q) for s in cand]
            assert abs(d[k] - min(dist)) <= 1e-13 * diag_of(Q)


def test_projection_brute_force_tiny():
    rng = np.random.default_rng(23)
    curves = [rand_curve(rng, p, n, repeat=0.3) for p, n in ((2, 4), (4, 6), (7, 9))]
    cs = synth.pack_curves([2, 4, 7], [c[0] for c in curves], [c[1] for c in curves])
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        sp = scipy_curve(p, U, P)
        ts = np.linspace(0, 1, 1_000_001)
        pts = sp(ts)
        qs = rng.uniform(-0.2, 1.2, (34, 3))
        t, d = O.project_curves(cs, np.full(len(qs), c, np.int32), qs)
        for k, q in enumerate(qs):
            D = np.sum((pts - q) ** 2, axis=1)
            loc = np.where((D[1:-1] <= D[:-2]) & (D[1:-1] <= D[2:]))[0] + 1
            loc = np.concatenate([[0, len(D) - 1], loc])
            best = np.inf
            for j in loc[np.argsort(D[loc])[:4]]:
                lo, hi = ts[max(j - 1, 0)], ts[min(j + 1, len(ts) - 1)]
                r = minimize_scalar(lambda s: np.sum((sp(s) - q) ** 2), bounds=(lo, hi), method="bounded",
                                    options={"xatol": 1e-13})
                best = min(best, np.sqrt(r.fun), np.sqrt(D[j]))
            assert d[k] <= best + 1e-13 * diag_of(P)
            assert d[k] >= best - 1e-9 * diag_of(P)


def test_inversion_round_trip():
    cs, qs = synth.curve_set(seed=24, n_curves=12, n_proj=10, n_inv=600)
    C, _, _ = O.eval_curves(cs, qs.inv_curve, qs.inv_t)
    t, d = O.project_curves(cs, qs.inv_curve, C)
    diag = O.curve_diag(cs)[qs.inv_curve]
    assert np.all(d <= 1e-13 * diag)
    # the recovered parameter maps back onto the same point
    C2, _, _ = O.eval_curves(cs, qs.inv_curve, t)
    assert np.all(np.linalg.norm(C2 - C, axis=1) <= 1e-13 * diag)


# ------------------------------------------------------------ surfaces

def _rand_surface(rng, pu, pv, nu, nv):
    U = synth.random_clamped_knots(rng, pu, nu, 0.2)
    V = synth.random_clamped_knots(rng, pv, nv, 0.2)
    P = synth._sinusoid_net(rng, nu, nv)
    return U, V, P


@pytest.mark.parametrize("pu,pv", [(1, 1), (2, 3), (3, 5), (5, 4)])
def test_surface_eval_matches_scipy(pu, pv):
    rng = np.random.default_rng(700 + 10 * pu + pv)
    U, V, P = _rand_surface(rng, pu, pv, 9, 10)
    ss = synth.pack_surfaces([pu], [pv], [U], [V], [P])
    uv = rng.uniform(0, 1, (100, 2))
    out = O.eval_surfaces(ss, np.zeros(100, np.int32), uv)
    for k in range(100):
        u, v = uv[k]
        ref = [scipy_surface(pu, pv, U, V, P, u, v, du, dv) for du, dv in ((0, 0), (1, 0), (0, 1))]
        for r, o in zip(ref, out[:3]):
            assert np.abs(o[k] - r).max() <= 1e-11 * (1 + np.abs(r).max())
        if pu >= 2 and pv >= 1:
            r = scipy_surface(pu, pv, U, V, P, u, v, 1, 1)
            assert np.abs(out[4][k] - r).max() <= 1e-9 * (1 + np.abs(r).max())


@pytest.mark.parametrize("pu,pv,tol", [(2, 3, 0.0), (4, 2, 1e-6), (5, 4, 1e-3)])
def test_surface_decomposition_meets_tolerance(pu, pv, tol):
    rng = np.random.default_rng(800 + pu * 10 + pv)
    U, V, P = _rand_surface(rng, pu, pv, 7, 6)
    ss = synth.pack_surfaces([pu], [pv], [U], [V], [P])
    d = O.decompose_surfaces(ss, tol)
    assert d.status == O.OK
    thr = tol * diag_of(P)
    if pu <= 3 and pv <= 3:
        nsp = sum(U[a] < U[a + 1] for a in range(pu, 7)) * sum(V[b] < V[b + 1] for b in range(pv, 6))
        assert d.total == nsp
    area = np.sum((d.prange[:, 1] - d.prange[:, 0]) * (d.prange[:, 3] - d.prange[:, 2]))
    assert abs(area - 1.0) <= 1e-12
    for k in rng.choice(d.total, size=min(d.total, 60), replace=False):
        u0, u1, v0, v1 = d.prange[k]
        for a, b in rng.uniform(0, 1, (5, 2)):
            ref = scipy_surface(pu, pv, U, V, P, u0 + a * (u1 - u0), v0 + b * (v1 - v0))
            got = bez_patch(d.ctrl[k], a, b)
            assert np.linalg.norm(got - ref) <= thr + 1e-13


def test_surface_projection_onto_planar_rectangle():
    """A (3,2)-degree surface with Greville nets is the rectangle
    o + R (u Lx, v Ly, 0) (bilinear precision): closed-form projection."""
    rng = np.random.default_rng(25)
    pu, pv, nu, nv = 3, 2, 7, 6
    U = synth.random_clamped_knots(rng, pu, nu, 0.0)
    V = synth.random_clamped_knots(rng, pv, nv, 0.0)
    Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    o, Lx, Ly = rng.uniform(-1, 1, 3), 1.3, 0.7
    gu, gv = greville(U, pu, nu), greville(V, pv, nv)
    P = np.array([[o + Rm @ np.array([a * Lx, b * Ly, 0.0]) for b in gv] for a in gu])
    ss = synth.pack_surfaces([pu], [pv], [U], [V], [P])
    qs = o + rng.uniform(-1, 2, (80, 3))
    uv, d = O.project_surfaces(ss, np.zeros(80, np.int32), qs)
    loc = (qs - o) @ Rm
    us = np.clip(loc[:, 0] / Lx, 0, 1)
    vs = np.clip(loc[:, 1] / Ly, 0, 1)
    ref = np.linalg.norm(loc - np.stack([us * Lx, vs * Ly, 0 * us], 1), axis=1)
    assert np.abs(d - ref).max() <= 1e-13 * 4
    inside = (us > 1e-6) & (us < 1 - 1e-6) & (vs > 1e-6) & (vs < 1 - 1e-6)
    assert np.abs(uv[inside, 0] - us[inside]).max() <= 1e-7
    assert np.abs(uv[inside, 1] - vs[inside]).max() <= 1e-7


def test_surface_projection_brute_force_tiny():
    rng = np.random.default_rng(26)
    pu, pv = 3, 2
    U, V, P = _rand_surface(rng, pu, pv, 5, 4)
    ss = synth.pack_surfaces([pu], [pv], [U], [V], [P])
    qs = P.reshape(-1, 3).mean(0) + rng.uniform(-0.6, 0.6, (16, 3))
    uv, d = O.project_surfaces(ss, np.zeros(len(qs), np.int32), qs)
    g = np.linspace(0, 1, 301)
    bu, bv = BSpline(U, np.eye(5), pu)(g), BSpline(V, np.eye(4), pv)(g)
    grid = np.einsum("ai,bj,ijc->abc", bu, bv, P)
    for k, q in enumerate(qs):
        D = np.sum((grid - q) ** 2, axis=2)
        flat = np.argsort(D.ravel())[:6]
        best = np.sqrt(D.ravel()[flat[0]])
        for f in flat:
            a, b = divmod(int(f), len(g))
            r = minimize(lambda x: np.sum((scipy_surface(pu, pv, U, V, P, x[0], x[1]) - q) ** 2),
                         x0=[g[a], g[b]], bounds=[(0, 1), (0, 1)], method="L-BFGS-B",
                         options={"ftol": 1e-15, "gtol": 1e-12})
            best = min(best, np.sqrt(r.fun))
        assert d[k] <= best + 1e-9 * diag_of(P)
        assert d[k] >= best - 1e-6 * diag_of(P)


def test_surface_inversion_round_trip():
    rng = np.random.default_rng(27)
    U, V, P = _rand_surface(rng, 4, 3, 9, 8)
    ss = synth.pack_surfaces([4], [3], [U], [V], [P])
    uv0 = rng.uniform(0, 1, (60, 2))
    S = O.eval_surfaces(ss, np.zeros(60, np.int32), uv0)[0]
    uv, d = O.project_surfaces(ss, np.zeros(60, np.int32), S)
    assert np.all(d <= 1e-12 * diag_of(P))
