"""Pins of the oracle's rational-surface functions (evaluation, derivative
bounds, projection on the original surface) against facts fixed by
mathematics:

* evaluation against SciPy's B-spline basis matrices (tensor sums of the
  numerator and of the weight, divided);
* on exact NURBS cylinders: the radius, S_v along the axis, S_uv = S_vv = 0,
  the tangent condition and the circle's curvature identity, and the
  closed-form distance of the projection;
* partial derivatives against central differences;
* the per-span-pair derivative bounds the branch and bound rests on, against
  sampled derivatives;
* projection never worse than a dense sample grid;
* equal weights give the non-rational results.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import oracle as O
from paper_2504_11498_gb300 import synth


def basis_matrix(U, p, x):
    return BSpline.design_matrix(np.clip(x, U[p], np.nextafter(U[-p - 1], -np.inf)), U, p).toarray()


def scipy_rational(ss, s, uv):
    pu, pv, U, V, P = ss.surface(s)
    w = ss.surface_weights(s)
    Bu, Bv = basis_matrix(U, pu, uv[:, 0]), basis_matrix(V, pv, uv[:, 1])
    num = np.einsum("ki,kj,ijc->kc", Bu, Bv, P * w[:, :, None])
    den = np.einsum("ki,kj,ij->k", Bu, Bv, w)
    return num / den[:, None]


def test_rational_surface_eval_matches_scipy():
    ss, _ = synth.nurbs_surface_set(n_surf=6, n_proj=1, w_range=(0.25, 4.0))
    uv = np.random.default_rng(1).uniform(0.0, 1.0, size=(400, 2))
    for s in range(ss.n):
        got = O.eval_surfaces(ss, np.full(len(uv), s, np.int32), uv)[0]
        assert np.abs(got - scipy_rational(ss, s, uv)).max() <= 1e-14, s


def test_cylinder_geometry_and_derivative_identities():
    ss, _, _, centre, axis, radius, height = synth.nurbs_cylinders(n_surf=6, n_proj=1)
    uv = np.random.default_rng(2).uniform(0.0, 1.0, size=(500, 2))
    for s in range(ss.n):
        S, Su, Sv, Suu, Suv, Svv = O.eval_surfaces(ss, np.full(len(uv), s, np.int32), uv)
        d = S - centre[s]
        h = d @ axis[s]
        rad = d - h[:, None] * axis[s]
        r = radius[s]
        assert np.abs(np.linalg.norm(rad, axis=1) - r).max() <= 1e-14
        assert np.allclose(h, uv[:, 1] * height[s], atol=1e-14)
        assert np.abs(Sv - height[s] * axis[s]).max() <= 1e-13
        assert np.abs(Suv).max() <= 1e-12 and np.abs(Svv).max() <= 1e-12
        sp = np.linalg.norm(Su, axis=1)
        assert np.abs(np.einsum("ij,ij->i", rad, Su)).max() <= 1e-13 * r * sp.max()
        assert np.abs(Su @ axis[s]).max() <= 1e-13 * sp.max()
        # the circle's curvature: (S - axis point).S_uu = -|S_u|^2
        assert np.allclose(np.einsum("ij,ij->i", rad, Suu), -sp ** 2, rtol=1e-11, atol=1e-11 * sp.max() ** 2)


def test_rational_partials_finite_differences():
    ss, _ = synth.nurbs_surface_set(seed=10, n_surf=4, n_proj=1, deg_range=(2, 4), n_range=(6, 9))
    rng = np.random.default_rng(3)
    h = 1e-6
    for s in range(ss.n):
        pu, pv, U, V, _ = ss.surface(s)
        inner_u = np.unique(U[(U > 0) & (U < 1)])
        inner_v = np.unique(V[(V > 0) & (V < 1)])
        uv = rng.uniform(0.01, 0.99, size=(200, 2))
        keep = np.ones(len(uv), bool)
        if len(inner_u):
            keep &= np.min(np.abs(uv[:, :1] - inner_u[None, :]), axis=1) > 1e-3
        if len(inner_v):
            keep &= np.min(np.abs(uv[:, 1:] - inner_v[None, :]), axis=1) > 1e-3
        uv = uv[keep]
        idx = np.full(len(uv), s, np.int32)
        S, Su, Sv, Suu, Suv, Svv = O.eval_surfaces(ss, idx, uv)
        up, um = O.eval_surfaces(ss, idx, uv + [h, 0]), O.eval_surfaces(ss, idx, uv - [h, 0])
        vp, vm = O.eval_surfaces(ss, idx, uv + [0, h]), O.eval_surfaces(ss, idx, uv - [0, h])
        sc1 = 1.0 + max(np.abs(Su).max(), np.abs(Sv).max())
        sc2 = 1.0 + max(np.abs(Suu).max(), np.abs(Suv).max(), np.abs(Svv).max())
        assert np.abs((up[0] - um[0]) / (2 * h) - Su).max() <= 1e-6 * (sc1 + sc2)
        assert np.abs((vp[0] - vm[0]) / (2 * h) - Sv).max() <= 1e-6 * (sc1 + sc2)
        assert np.abs((up[1] - um[1]) / (2 * h) - Suu).max() <= 1e-5 * sc2
        assert np.abs((vp[1] - vm[1]) / (2 * h) - Suv).max() <= 1e-5 * sc2
        assert np.abs((vp[2] - vm[2]) / (2 * h) - Svv).max() <= 1e-5 * sc2


def heavy_weight_patches(seed=14, n=6):
    """Biquadratic and bicubic single-span patches with one heavy interior
    weight (10..100 x the others): the surface is pulled toward that point
    and its parameterisation is driven by the weight's variation."""
    rng = np.random.default_rng(seed)
    deg, KU, KV, nets, ws = [], [], [], [], []
    for k in range(n):
        p = 2 + k % 2
        P = rng.uniform(0.0, 1.0, size=(p + 1, p + 1, 3))
        w = np.ones((p + 1, p + 1))
        w[1 + k % (p - 1), 1] = rng.uniform(10.0, 100.0)
        deg.append(p)
        KU.append(synth.uniform_clamped_knots(p, p + 1))
        KV.append(synth.uniform_clamped_knots(p, p + 1))
        nets.append(P)
        ws.append(w)
    return synth.pack_surfaces(deg, deg, KU, KV, nets, ws)


def extreme_weight_patches(n=120):
    """Single-span patches of degrees 1..3 with weights log-uniform over
    [0.01, 100] (patch k drawn with seed k): where the weight's variation
    carries the derivative, so that every term of the bound is needed."""
    deg, KU, nets, ws = [], [], [], []
    for k in range(n):
        rng = np.random.default_rng(k)
        p = int(rng.integers(1, 4))
        nets.append(rng.uniform(0, 1, size=(p + 1, p + 1, 3)))
        ws.append(np.exp(rng.uniform(np.log(0.01), np.log(100.0), size=(p + 1, p + 1))))
        deg.append(p)
        KU.append(synth.uniform_clamped_knots(p, p + 1))
    return synth.pack_surfaces(deg, deg, KU, KU, nets, ws)


@pytest.mark.parametrize("which", ["random", "heavy", "extreme"])
def test_rational_derivative_bounds_cover_samples(which):
    if which == "random":
        ss, _ = synth.nurbs_surface_set(seed=11, n_surf=4, n_proj=1, deg_range=(2, 4), n_range=(6, 9),
                                        w_range=(0.25, 4.0))
    elif which == "heavy":
        ss = heavy_weight_patches()
    else:
        ss = extreme_weight_patches()
    g = np.linspace(0.0, 1.0, 41)
    ratios = []
    for s in range(ss.n):
        pu, pv, U, V, P = ss.surface(s)
        w = ss.surface_weights(s)
        for qu in range(pu, P.shape[0]):
            if not U[qu] < U[qu + 1]:
                continue
            for qv in range(pv, P.shape[1]):
                if not V[qv] < V[qv + 1]:
                    continue
                Vu, Vv, Auu, Avv = O.surf_deriv_bounds(pu, pv, U, V, P, w, qu, qv)
                # the closed span pair, approached from inside at the far ends
                gu = np.minimum(U[qu] + g * (U[qu + 1] - U[qu]), np.nextafter(U[qu + 1], -np.inf))
                gv = np.minimum(V[qv] + g * (V[qv + 1] - V[qv]), np.nextafter(V[qv + 1], -np.inf))
                uu, vv = np.meshgrid(gu, gv, indexing="ij")
                uv = np.stack([uu.ravel(), vv.ravel()], 1)
                _, Su, Sv, Suu, _, Svv = O.eval_surfaces(ss, np.full(len(uv), s, np.int32), uv)
                got = [np.linalg.norm(x, axis=1).max() for x in (Su, Sv, Suu, Svv)]
                for m, b in zip(got, (Vu, Vv, Auu, Avv)):
                    assert m <= b * (1 + 1e-12), (s, qu, qv, m, b)
                ratios.append(Vu / got[0])
    # loose by the weights' range and the convex-hull radius, but bounded
    if which != "extreme":
        assert np.median(ratios) < 100.0, np.median(ratios)
    if which == "heavy":
        # the sampled derivatives come close to the bounds: a bound that
        # dropped a term would fall below them
        assert min(ratios) < 4.0, min(ratios)


def test_cylinder_projection_closed_form():
    ss, q, sidx, centre, axis, radius, _ = synth.nurbs_cylinders(n_surf=8, n_proj=1500)
    uv, d = O.project_surfaces(ss, sidx, q)
    dq = q - centre[sidx]
    hq = np.einsum("ij,ij->i", dq, axis[sidx])
    rq = np.linalg.norm(dq - hq[:, None] * axis[sidx], axis=1)
    assert np.abs(d - np.abs(rq - radius[sidx])).max() <= 1e-13
    # the foot point is at the query's height, to the conditioning of a
    # parameter at a minimum of D (about sqrt(FP64 rounding) x d)
    S = O.eval_surfaces(ss, sidx, uv)[0]
    ds = S - centre[sidx]
    assert np.all(np.abs(np.einsum("ij,ij->i", ds, axis[sidx]) - hq) <= 1e-7 * np.maximum(d, 1e-3))


def test_rational_projection_no_worse_than_dense_grid():
    ss, sq = synth.nurbs_surface_set(seed=12, n_surf=3, n_proj=90, deg_range=(2, 3), n_range=(6, 8),
                                     w_range=(0.25, 4.0))
    diag = O.surface_diag(ss)
    q = O.eval_surfaces(ss, sq.proj_surf, sq.proj_uv)[0] + sq.proj_dir * sq.proj_r[:, None]
    _, d = O.project_surfaces(ss, sq.proj_surf, q)
    g = np.linspace(0.0, 1.0, 401)
    uu, vv = np.meshgrid(g, g, indexing="ij")
    grid = np.stack([uu.ravel(), vv.ravel()], 1)
    for s in range(ss.n):
        S = O.eval_surfaces(ss, np.full(len(grid), s, np.int32), grid)[0]
        for k in np.where(sq.proj_surf == s)[0]:
            brute = np.sqrt(((S - q[k]) ** 2).sum(1)).min()
            assert d[k] <= brute + 1e-15, (s, k, d[k], brute)
            assert brute - d[k] <= 2e-3 * diag[s], (s, k, d[k], brute)


def test_equal_weights_give_non_rational_surfaces():
    ss, sq = synth.surface_set(seed=13, n_surf=3, n_proj=60, n_inv=0, deg_range=(2, 3), n_range=(6, 9))
    rat = synth.SurfaceSet(ss.deg_u, ss.deg_v, ss.n_u, ss.n_v, ss.knot_u_off, ss.knots_u, ss.knot_v_off,
                           ss.knots_v, ss.cp_off, ss.cps, np.full(len(ss.cps), 1.7))
    uv = np.random.default_rng(4).uniform(0, 1, (300, 2))
    idx = np.random.default_rng(5).integers(0, ss.n, 300).astype(np.int32)
    for a, b in zip(O.eval_surfaces(ss, idx, uv), O.eval_surfaces(rat, idx, uv)):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)
    q = O.eval_surfaces(ss, sq.proj_surf, sq.proj_uv)[0] + sq.proj_dir * sq.proj_r[:, None]
    _, d0 = O.project_surfaces(ss, sq.proj_surf, q)
    _, d1 = O.project_surfaces(rat, sq.proj_surf, q)
    assert np.allclose(d0, d1, rtol=1e-12, atol=1e-14)


# ------------------------------------------------- homogeneous decomposition

def rbez2(H, u, v):
    """Explicit rational tensor Bernstein sum of the homogeneous net H
    [pu+1][pv+1][4] at parameter arrays u, v of equal length."""
    import math
    H = np.asarray(H)
    pu, pv = H.shape[0] - 1, H.shape[1] - 1
    u, v = np.atleast_1d(u), np.atleast_1d(v)
    Bu = np.stack([math.comb(pu, i) * u ** i * (1 - u) ** (pu - i) for i in range(pu + 1)], 1)
    Bv = np.stack([math.comb(pv, j) * v ** j * (1 - v) ** (pv - j) for j in range(pv + 1)], 1)
    S = np.einsum("ki,kj,ijc->kc", Bu, Bv, H)
    return S[:, :3] / S[:, 3:]


def bicubic(R, u, v):
    import math
    Bu = np.stack([math.comb(3, i) * u ** i * (1 - u) ** (3 - i) for i in range(4)], 1)
    Bv = np.stack([math.comb(3, j) * v ** j * (1 - v) ** (3 - j) for j in range(4)], 1)
    return np.einsum("ki,kj,ijc->kc", Bu, Bv, R)


def random_rnet(rng, pu, pv, wlo=0.2, whi=5.0):
    P = rng.uniform(-1, 1, size=(pu + 1, pv + 1, 3))
    w = np.exp(rng.uniform(np.log(wlo), np.log(whi), size=(pu + 1, pv + 1)))
    return np.concatenate([P * w[..., None], w[..., None]], axis=2)


def test_bicubic_hermite_matches_corner_values_partials_twists():
    rng = np.random.default_rng(31)
    h = 1e-5
    for pu in range(1, 5):
        for pv in range(1, 5):
            H = random_rnet(rng, pu, pv)
            R = O.rsurf_hermite(H)
            for cu in (0.0, 1.0):
                for cv in (0.0, 1.0):
                    su, sv = (1.0 if cu == 0 else -1.0), (1.0 if cv == 0 else -1.0)
                    i0, i1 = (0, 1) if cu == 0 else (3, 2)
                    j0, j1 = (0, 1) if cv == 0 else (3, 2)
                    f = lambda du, dv: rbez2(H, np.array([cu + su * du]), np.array([cv + sv * dv]))[0]
                    assert np.allclose(R[i0, j0], f(0, 0), atol=1e-14)
                    # one-sided second-order differences into the piece
                    fu = (-3 * f(0, 0) + 4 * f(h, 0) - f(2 * h, 0)) / (2 * h)
                    fv = (-3 * f(0, 0) + 4 * f(0, h) - f(0, 2 * h)) / (2 * h)
                    # second-order one-sided stencil in both directions
                    cst = (-3.0, 4.0, -1.0)
                    fuv = sum(cst[a] * cst[b] * f(a * h, b * h) for a in range(3) for b in range(3)) / (4 * h * h)
                    sc = 1 + np.abs(fu).max() + np.abs(fv).max()
                    assert np.abs(3 * (R[i1, j0] - R[i0, j0]) - fu).max() <= 1e-5 * sc, (pu, pv, cu, cv)
                    assert np.abs(3 * (R[i0, j1] - R[i0, j0]) - fv).max() <= 1e-5 * sc, (pu, pv, cu, cv)
                    twist = 9 * (R[i1, j1] - R[i1, j0] - R[i0, j1] + R[i0, j0])
                    assert np.abs(twist - fuv).max() <= 1e-4 * (1 + np.abs(fuv).max()), (pu, pv, cu, cv)


def test_surface_bound_covers_sampled_deviation():
    rng = np.random.default_rng(32)
    g = np.linspace(0.0, 1.0, 41)
    uu, vv = np.meshgrid(g, g, indexing="ij")
    u, v = uu.ravel(), vv.ravel()
    for pu in range(1, 5):
        for pv in range(1, 5):
            for _ in range(4):
                H = random_rnet(rng, pu, pv)
                R = O.rsurf_hermite(H)
                b2 = O.rsurf_bound2(H, R)
                dev = np.linalg.norm(rbez2(H, u, v) - bicubic(R, u, v), axis=1).max()
                assert dev ** 2 <= b2 * (1 + 1e-9) + 1e-28, (pu, pv, dev, np.sqrt(b2))
    # the net scaled by a constant is the same surface: same patch, same bound
    for pu, pv in ((1, 1), (2, 3), (4, 2)):
        H = random_rnet(rng, pu, pv)
        R = O.rsurf_hermite(H)
        for lam in (1e-2, 1e3):
            assert np.allclose(O.rsurf_hermite(lam * H), R, rtol=1e-12, atol=1e-13)
            assert np.isclose(O.rsurf_bound2(lam * H, R), O.rsurf_bound2(H, R), rtol=1e-9)
    # a polynomial piece of degree <= 3 is its own Hermite patch: bound ~0
    for pu, pv in ((1, 2), (3, 3), (2, 3)):
        P = rng.uniform(-1, 1, size=(pu + 1, pv + 1, 3))
        H = np.concatenate([2.0 * P, np.full((pu + 1, pv + 1, 1), 2.0)], axis=2)
        R = O.rsurf_hermite(H)
        assert O.rsurf_bound2(H, R) <= 1e-28
        assert np.abs(bicubic(R, u, v) - rbez2(H, u, v)).max() <= 1e-14


@pytest.mark.parametrize("which,tol", [("random", 1e-3), ("cylinders", 1e-7)])
def test_rational_surface_decomposition_within_tolerance(which, tol):
    if which == "random":
        ss, _ = synth.nurbs_surface_set(seed=15, n_surf=3, n_proj=1, deg_range=(2, 3), n_range=(5, 7))
    else:
        ss = synth.nurbs_cylinders(seed=16, n_surf=3, n_proj=1)[0]
    dec = O.decompose_surfaces(ss, tol)
    assert dec.status == 0
    diag = O.surface_diag(ss)
    g = np.linspace(0.0, 1.0, 9)
    uu, vv = np.meshgrid(g, g, indexing="ij")
    u, v = uu.ravel(), vv.ravel()
    worst = 0.0
    for s in range(ss.n):
        area = 0.0
        for k in range(dec.seg_off[s], dec.seg_off[s + 1]):
            u0, u1, v0, v1 = dec.prange[k]
            area += (u1 - u0) * (v1 - v0)
            S = O.eval_surfaces(ss, np.full(len(u), s, np.int32),
                                np.stack([u0 + u * (u1 - u0), v0 + v * (v1 - v0)], 1))[0]
            worst = max(worst, np.linalg.norm(S - bicubic(dec.ctrl[k], u, v), axis=1).max() / (tol * diag[s]))
        assert abs(area - 1.0) <= 1e-12  # the patches tile the domain
    assert worst <= 1.0 + 1e-9, worst


def test_equal_weights_decompose_as_non_rational():
    ss, _ = synth.surface_set(seed=17, n_surf=3, n_proj=1, n_inv=0, deg_range=(2, 4), n_range=(6, 8))
    rat = synth.SurfaceSet(ss.deg_u, ss.deg_v, ss.n_u, ss.n_v, ss.knot_u_off, ss.knots_u, ss.knot_v_off,
                           ss.knots_v, ss.cp_off, ss.cps, np.full(len(ss.cps), 3.0))
    d0, d1 = O.decompose_surfaces(ss, 1e-4), O.decompose_surfaces(rat, 1e-4)
    assert np.array_equal(d0.seg_off, d1.seg_off)
    assert np.array_equal(d0.ctrl, d1.ctrl) and np.array_equal(d0.prange, d1.prange)
