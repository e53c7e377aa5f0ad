"""Pins of the FP64 reference of the learned seed (oracle/mlp.py) against
facts that do not come from its own formulas: finite differences, the
Gaussian CDF, Adam's closed-form first step, invariances of the features,
brute force and closed forms for the segment minimiser."""
import math

import numpy as np
import pytest
from scipy import optimize, special

from oracle import mlp as M


def tiny_params(rng, widths=(5, 4, 3, 2)):
    p = {}
    for i in range(3):
        p[f"W{i + 1}"] = rng.normal(0, 0.8, (widths[i + 1], widths[i]))
        p[f"b{i + 1}"] = rng.normal(0, 0.3, widths[i + 1])
    p["w4"] = rng.normal(0, 0.8, widths[3])
    p["b4"] = rng.normal(0, 0.3, 1)
    return p


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = tiny_params(rng)
    X = rng.normal(0, 1, (7, 5))
    y = rng.uniform(0, 1, 7)
    _, g = M.loss_and_grads(p, X, y)
    h = 1e-6
    for name, arr in p.items():
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            lp = M.loss_and_grads(p, X, y)[0]
            arr[idx] = old - h
            lm = M.loss_and_grads(p, X, y)[0]
            arr[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[name], num, rtol=1e-5, atol=1e-9), name


def test_gelu_symmetry_and_gaussian_cdf():
    x = np.linspace(-8, 8, 4001)
    assert M.gelu(0.0) == 0.0
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)
    # the tanh form approximates x Phi(x) to a few 1e-4
    assert np.max(np.abs(M.gelu(x) - x * special.ndtr(x))) < 1e-3
    h = 1e-6
    assert np.allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), atol=1e-8)


def test_sigmoid_output_with_zero_weights():
    p = {k: np.zeros(s) for k, s in M._SHAPES}
    p["b4"] = np.array([0.7])
    t, _, _ = M.forward(p, np.ones((3, M.IN)))
    assert np.allclose(t, 1 / (1 + math.exp(-0.7)))


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0, 3, 5000), rng.normal(0, 1e-3, 1000), [0.0, 1.0, -2.5, 1 + 2 ** -8, 1 + 3 * 2 ** -8]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.round_bf16(x), ref)


def test_pack_layout():
    sizes = [int(np.prod(s)) for _, s in M._SHAPES]
    assert sum(sizes) + 3 == M.NPARAM
    theta = np.arange(M.NPARAM, dtype=np.float64)
    p = M.unpack(theta)
    assert p["W1"][1, 0] == 16 and p["b1"][0] == 128 * 16 and p["b4"][0] == M.NPARAM - 4
    assert np.array_equal(M.pack(p)[:-3], theta[:-3])


def test_adam_first_step_and_convergence():
    rng = np.random.default_rng(1)
    g = rng.normal(size=10)
    th = rng.normal(size=10)
    new, m, v = M.adam(th, g, np.zeros(10), np.zeros(10), 1, 0.01)
    # bias correction makes the first step -lr g / (|g| + eps)
    assert np.allclose(new - th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    a = rng.normal(size=10)
    x, m, v = np.zeros(10), np.zeros(10), np.zeros(10)
    for k in range(1, 3001):
        x, m, v = M.adam(x, x - a, m, v, k, 0.01)
    assert np.max(np.abs(x - a)) < 1e-3


def test_features_invariances():
    rng = np.random.default_rng(2)
    P = rng.uniform(-1, 1, (50, 4, 3))
    q = rng.uniform(-2, 2, (50, 3))
    X = M.features(P, q)
    sh = rng.normal(size=3)
    assert np.allclose(M.features(P + sh, q + sh), X, atol=1e-12)
    assert np.allclose(M.features(3.7 * P, 3.7 * q), X, atol=1e-12)
    pts = X[:, :12].reshape(-1, 4, 3)
    ext = pts.max(1) - pts.min(1)
    assert np.allclose(ext.max(1), 1.0) and np.all(np.abs(pts) <= 0.5 + 1e-12)
    assert np.all(X[:, 15] == 0)


def test_features_query_split_along_and_across_the_chord():
    rng = np.random.default_rng(12)
    for _ in range(20):
        P = rng.uniform(-1, 1, (4, 3))
        ch = P[3] - P[0]
        d = ch / np.linalg.norm(ch)
        n = np.cross(d, rng.normal(size=3))
        n /= np.linalg.norm(n)
        lo, hi = P.min(0), P.max(0)
        c, s = 0.5 * (lo + hi), 1.0 / (hi - lo).max()
        lam = rng.uniform(-0.2, 1.2)
        # far across the chord: along-chord coordinate kept, across part unit length
        q = P[0] + lam * ch + 1e3 * n
        f = M.features(P[None], q[None])[0, 12:15]
        a = ((P[0] + lam * ch - c) * s) @ d
        assert abs(f @ d - a) < 1e-9
        assert abs(np.linalg.norm(f - (f @ d) * d) - 1.0) < 1e-9
        assert (f - (f @ d) * d) @ n > 0.999
        # close to the segment the query coordinates are unchanged
        qn = c + 0.3 / s * rng.uniform(-1, 1, 3) / np.sqrt(3)
        assert np.allclose(M.features(P[None], qn[None])[0, 12:15], (qn - c) * s, atol=1e-12)


def test_segment_minimiser_line_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, b = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
        P = np.array([a + (b - a) * k / 3 for k in range(4)])  # linear parametrisation
        q = rng.uniform(-1.5, 1.5, 3)
        u_ref = np.clip((q - a) @ (b - a) / ((b - a) @ (b - a)), 0, 1)
        u, D = M.segment_minimiser(P, q)
        assert abs(u - u_ref) < 1e-9
        assert abs(D - np.sum((a + u_ref * (b - a) - q) ** 2)) < 1e-14


def test_segment_minimiser_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(25):
        P = rng.uniform(-1, 1, (4, 3))
        q = rng.uniform(-1, 1, 3)
        u, D = M.segment_minimiser(P, q)

        def f(x):
            return float(np.sum((M._bezier(P, np.array([x]))[0] - q) ** 2))

        best = min(f(0.0), f(1.0))
        grid = np.linspace(0, 1, 201)
        for lo, hi in zip(grid[:-1], grid[1:]):
            r = optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12})
            best = min(best, r.fun)
        assert D <= best + 1e-13
        assert abs(D - f(u)) < 1e-15


def test_segment_minimiser_tie_takes_smaller_u():
    P = np.array([[-1.0, 0, 0], [-0.5, -1, 0], [0.5, -1, 0], [1, 0, 0]])
    u, D = M.segment_minimiser(P, np.array([0.0, 5.0, 0.0]))
    assert u == 0.0 and D == pytest.approx(26.0)


# ------------------------------------------------------- surface network

def test_two_output_gradients_match_central_differences():
    """The surface network's head (two sigmoid outputs, loss averaged over
    rows and outputs) by the chain rule vs central differences."""
    rng = np.random.default_rng(3)
    p = tiny_params(rng, widths=(6, 4, 3, 3))
    del p["w4"]
    p["W4"] = rng.normal(0, 0.8, (2, 3))
    p["b4"] = rng.normal(0, 0.3, 2)
    X = rng.normal(0, 1, (5, 6))
    y = rng.uniform(0, 1, (5, 2))
    loss, g = M.loss_and_grads(p, X, y)
    t, _, _ = M.forward(p, X)
    assert t.shape == (5, 2) and np.isclose(loss, np.mean((t - y) ** 2))
    h = 1e-6
    for name, arr in p.items():
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            lp = M.loss_and_grads(p, X, y)[0]
            arr[idx] = old - h
            lm = M.loss_and_grads(p, X, y)[0]
            arr[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[name], num, rtol=1e-5, atol=1e-9), name


def test_surface_layout_round_trip():
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 1, M.SNPARAM)
    theta[-2:] = 0.0
    p = M.unpack(theta, M.SHAPES_SURF)
    assert p["W1"].shape == (128, 64) and p["W4"].shape == (2, 128) and p["b4"].shape == (2,)
    assert np.array_equal(M.pack(p, M.SNPARAM, M.SHAPES_SURF), theta)


def _flat_patch(rng):
    """A bicubic whose net is an affine image of the unit square (bilinear
    precision): S(u, v) = o + u A + v B exactly."""
    o, A, B = rng.normal(0, 1, 3), rng.normal(0, 1, 3), rng.normal(0, 1, 3)
    g = np.arange(4) / 3.0
    P = o + g[:, None, None] * A + g[None, :, None] * B
    return P, o, A, B


def test_patch_minimiser_flat_patch_closed_form():
    """On a flat parallelogram the minimiser is the projection onto its
    plane, clamped to the square: a small convex QP solved here by SciPy."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        P, o, A, B = _flat_patch(rng)
        q = o + rng.uniform(-0.5, 1.5) * A + rng.uniform(-0.5, 1.5) * B + rng.normal(0, 1, 3)
        res = optimize.minimize(lambda x: np.sum((o + x[0] * A + x[1] * B - q) ** 2), x0=[0.5, 0.5],
                                bounds=[(0, 1), (0, 1)], method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-12})
        u, v, D = M.patch_minimiser(P, q)
        assert D <= res.fun + 1e-12
        assert np.allclose([u, v], res.x, atol=1e-6)


def test_patch_minimiser_point_on_patch_and_brute_force():
    rng = np.random.default_rng(6)
    for _ in range(6):
        P = rng.uniform(0, 1, (4, 4, 3))
        u0, v0 = rng.uniform(0, 1, 2)
        q = M._patch(P, u0, v0)
        u, v, D = M.patch_minimiser(P, q)
        assert D <= 1e-24
        # a random point: no sample of a 401 x 401 grid is closer
        q = rng.uniform(-0.5, 1.5, 3)
        u, v, D = M.patch_minimiser(P, q)
        g = np.linspace(0, 1, 401)
        uu, vv = np.meshgrid(g, g, indexing="ij")
        Dg = ((M._patch(P, uu, vv) - q) ** 2).sum(axis=-1)
        assert D <= Dg.min() + 1e-15
        assert np.isclose(D, np.sum((M._patch(P, u, v) - q) ** 2), rtol=0, atol=1e-15)


def test_surface_features_invariances():
    """Translating or scaling the patch and the query together leaves the
    inputs unchanged; a query far along the frame's normal is clamped to the
    unit normal offset, its tangential part kept."""
    rng = np.random.default_rng(7)
    P = rng.uniform(0, 1, (3, 4, 4, 3))
    q = rng.uniform(-1, 2, (3, 3))
    X = M.surface_features(P, q)
    s, t = 3.7, rng.normal(0, 5, 3)
    assert np.allclose(M.surface_features(P * s + t, q * s + t), X, atol=1e-12)
    assert np.all(X[:, 51:] == 0)
    F, _, _, _ = _flat_patch(rng)
    e1 = F[3, 0] - F[0, 0]
    e1 /= np.linalg.norm(e1)
    w = F[0, 3] - F[0, 0]
    w -= (w @ e1) * e1
    e2 = w / np.linalg.norm(w)
    nn = np.cross(e1, e2)
    q0 = F[0, 0] + 0.3 * (F[3, 0] - F[0, 0])
    Xf = M.surface_features(np.stack([F, F]), np.stack([q0 + 50 * nn, q0 - 50 * nn]))
    for k, sign in ((0, 1), (1, -1)):
        assert np.isclose(Xf[k, 48:51] @ nn, sign)
    assert np.allclose(Xf[0, 48:51] - Xf[0, 48:51] @ nn * nn, Xf[1, 48:51] - Xf[1, 48:51] @ nn * nn)
