"""Seeded synthetic workloads (input generators only).

This module draws random B-spline curves, surfaces and query recipes with
NumPy's ``default_rng``.  It holds none of the method's arithmetic: it never
evaluates a spline, decomposes one or projects a point.  Points *on* a spline
(inversion queries, surface projection queries) are returned as parameters and
offsets; the caller evaluates them with whichever evaluator it is testing.

Both the CPU oracle tests and the GPU path consume these arrays, so the two
sides always see identical inputs.

Workloads (the shapes of the paper's experiments are curves of degree 4-6 with
5-50 control points, coordinates in [0, 1]; Sec. 5, Tables 1-2):

* ``single_cubic``   one clamped cubic, 16 control points ~U[-1,1]^3, uniform
                     knots (13 spans), 10k projection + 10k inversion queries.
* ``curve_set``      4,096 curves, degree ~U{2..7}, 8..64 control points in the
                     unit cube, clamped non-uniform knots with 10% repeated
                     interior knots; 1M + 1M queries.
* ``surface_set``    1,024 surfaces, bi-degree ~U{2..5}^2, 8..32 nets on a grid
                     with a sum-of-sinusoids height plus noise.
* ``ragged_mix``     65,536 cubic curves + 8,192 bicubic surfaces with
                     log-normal segment counts and Zipf(1.1) query skew.
* ``nurbs_curve_set`` the ``curve_set`` recipe with a positive weight per
                     control point, log-uniform in [1/2, 2] (rational curves).
* ``nurbs_circles``  full circles as rational quadratics (nine control
                     points on a square, corner weights sqrt(2)/2), random
                     centre, radius and plane.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CurveSet:
    """CSR-packed B-spline curves.

    degree[n] int32; knot_off[n+1] int64 into knots (float64);
    cp_off[n+1] int64 into cps (float64, [ncp][3]).  Curve c has
    cp_off[c+1]-cp_off[c] control points and that many + degree + 1 knots.
    weights: None (non-rational), or [ncp total] float64, one positive
    weight per control point (rational curves, NURBS).
    """

    degree: np.ndarray
    knot_off: np.ndarray
    knots: np.ndarray
    cp_off: np.ndarray
    cps: np.ndarray
    weights: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.degree.shape[0])

    def curve(self, c: int):
        p = int(self.degree[c])
        U = self.knots[self.knot_off[c]:self.knot_off[c + 1]]
        P = self.cps[self.cp_off[c]:self.cp_off[c + 1]]
        return p, U, P

    def curve_weights(self, c: int):
        return None if self.weights is None else self.weights[self.cp_off[c]:self.cp_off[c + 1]]

    def subset(self, idx) -> "CurveSet":
        idx = np.asarray(idx, dtype=np.int64)
        curves = [self.curve(int(c)) for c in idx]
        w = None if self.weights is None else [self.curve_weights(int(c)) for c in idx]
        return pack_curves([c[0] for c in curves], [c[1] for c in curves], [c[2] for c in curves], w)


@dataclass
class SurfaceSet:
    """CSR-packed tensor-product B-spline surfaces.

    deg_u, deg_v, n_u, n_v: [n] int32.  knot_u_off/knot_v_off [n+1] int64
    into knots_u/knots_v.  cp_off [n+1] int64 into cps, each surface's net
    stored row-major [n_u][n_v][3] (first index along u).  weights: None
    (non-rational), or [ncp total] float64, one positive weight per control
    point in the same order (rational surfaces).
    """

    deg_u: np.ndarray
    deg_v: np.ndarray
    n_u: np.ndarray
    n_v: np.ndarray
    knot_u_off: np.ndarray
    knots_u: np.ndarray
    knot_v_off: np.ndarray
    knots_v: np.ndarray
    cp_off: np.ndarray
    cps: np.ndarray
    weights: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.deg_u.shape[0])

    def surface_weights(self, s: int):
        """[n_u][n_v] weights of surface s, or None."""
        if self.weights is None:
            return None
        return self.weights[self.cp_off[s]:self.cp_off[s + 1]].reshape(int(self.n_u[s]), int(self.n_v[s]))

    def surface(self, s: int):
        U = self.knots_u[self.knot_u_off[s]:self.knot_u_off[s + 1]]
        V = self.knots_v[self.knot_v_off[s]:self.knot_v_off[s + 1]]
        P = self.cps[self.cp_off[s]:self.cp_off[s + 1]].reshape(int(self.n_u[s]), int(self.n_v[s]), 3)
        return int(self.deg_u[s]), int(self.deg_v[s]), U, V, P

    def subset(self, idx) -> "SurfaceSet":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.surface(int(s)) for s in idx]
        w = None if self.weights is None else [self.surface_weights(int(s)) for s in idx]
        return pack_surfaces(*zip(*parts), weight_list=w)


def pack_curves(degrees, knot_list, cp_list, weight_list=None) -> CurveSet:
    degrees = np.asarray(degrees, dtype=np.int32)
    klen = np.array([len(k) for k in knot_list], dtype=np.int64)
    clen = np.array([len(c) for c in cp_list], dtype=np.int64)
    knot_off = np.zeros(len(klen) + 1, dtype=np.int64)
    knot_off[1:] = np.cumsum(klen)
    cp_off = np.zeros(len(clen) + 1, dtype=np.int64)
    cp_off[1:] = np.cumsum(clen)
    knots = np.concatenate([np.asarray(k, dtype=np.float64) for k in knot_list]) if len(knot_list) else np.zeros(0)
    cps = (np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1, 3) for c in cp_list])
           if len(cp_list) else np.zeros((0, 3)))
    w = None
    if weight_list is not None:
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in weight_list])
                                 if len(weight_list) else np.zeros(0))
        assert w.shape == (len(cps),)
    return CurveSet(degrees, knot_off, np.ascontiguousarray(knots), cp_off, np.ascontiguousarray(cps), w)


def pack_surfaces(deg_u, deg_v, knots_u, knots_v, nets, weight_list=None) -> SurfaceSet:
    nets = [np.asarray(P, dtype=np.float64) for P in nets]
    n_u = np.array([P.shape[0] for P in nets], dtype=np.int32)
    n_v = np.array([P.shape[1] for P in nets], dtype=np.int32)

    def offs(lens):
        o = np.zeros(len(lens) + 1, dtype=np.int64)
        o[1:] = np.cumsum(lens)
        return o

    return SurfaceSet(
        np.asarray(deg_u, dtype=np.int32), np.asarray(deg_v, dtype=np.int32), n_u, n_v,
        offs([len(k) for k in knots_u]), np.concatenate([np.asarray(k, np.float64) for k in knots_u]),
        offs([len(k) for k in knots_v]), np.concatenate([np.asarray(k, np.float64) for k in knots_v]),
        offs([P.shape[0] * P.shape[1] for P in nets]),
        np.ascontiguousarray(np.concatenate([P.reshape(-1, 3) for P in nets])),
        None if weight_list is None else np.ascontiguousarray(
            np.concatenate([np.asarray(w, np.float64).reshape(-1) for w in weight_list])),
    )


# --------------------------------------------------------------------------
# knot vectors
# --------------------------------------------------------------------------

def uniform_clamped_knots(p: int, ncp: int) -> np.ndarray:
    """Clamped knots on [0,1] with ncp-p equal spans."""
    nint = ncp - p - 1
    inner = np.arange(1, nint + 1, dtype=np.float64) / (nint + 1)
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def random_clamped_knots(rng: np.random.Generator, p: int, ncp: int, repeat_prob: float = 0.1) -> np.ndarray:
    """Clamped knots on [0,1]: ncp-p-1 interior values sorted U(0,1); each is
    repeated, with probability repeat_prob, to a multiplicity ~U{2..p}; the
    expanded interior list is truncated to ncp-p-1 entries."""
    nint = ncp - p - 1
    vals = np.sort(rng.uniform(0.0, 1.0, size=nint))
    rep = rng.uniform(size=nint) < repeat_prob
    mult = rng.integers(2, max(p, 2) + 1, size=nint)
    expanded = []
    for v, r, m in zip(vals, rep, mult):
        expanded.extend([v] * (int(m) if (r and p >= 2) else 1))
    inner = np.array(expanded[:nint], dtype=np.float64)
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


# --------------------------------------------------------------------------
# curve workloads
# --------------------------------------------------------------------------

@dataclass
class CurveQueries:
    """Projection queries as points, inversion queries as parameters.

    proj_curve[np] int32, proj_xyz[np][3]; inv_curve[ni] int32, inv_t[ni]
    (the caller evaluates C(inv_t) to obtain the inversion points)."""

    proj_curve: np.ndarray
    proj_xyz: np.ndarray
    inv_curve: np.ndarray
    inv_t: np.ndarray


def cp_boxes(cs: CurveSet):
    """Per-curve axis-aligned box of the control points (lo, hi)."""
    lo = np.minimum.reduceat(cs.cps, cs.cp_off[:-1], axis=0)
    hi = np.maximum.reduceat(cs.cps, cs.cp_off[:-1], axis=0)
    return lo, hi


def _box_queries(rng, lo, hi, which, scale=1.2):
    c = 0.5 * (lo[which] + hi[which])
    h = 0.5 * scale * (hi[which] - lo[which])
    return c + h * rng.uniform(-1.0, 1.0, size=(len(which), 3))


def single_cubic(seed: int = 1, n_proj: int = 10_000, n_inv: int = 10_000):
    """One clamped cubic, 16 control points ~U[-1,1]^3, uniform knots (13 spans)."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(-1.0, 1.0, size=(16, 3))
    cs = pack_curves([3], [uniform_clamped_knots(3, 16)], [P])
    lo, hi = cp_boxes(cs)
    pc = np.zeros(n_proj, dtype=np.int32)
    q = _box_queries(rng, lo, hi, pc)
    ic = np.zeros(n_inv, dtype=np.int32)
    t = rng.uniform(0.0, 1.0, size=n_inv)
    return cs, CurveQueries(pc, q, ic, t)


def curve_set(seed: int = 2, n_curves: int = 4096, n_proj: int = 1_000_000, n_inv: int = 1_000_000,
              deg_range=(2, 7), ncp_range=(8, 64)):
    """Random curves: degree ~U{2..7}, 8..64 control points ~U[0,1]^3,
    clamped non-uniform knots; queries assigned uniformly to curves."""
    rng = np.random.default_rng(seed)
    degs = rng.integers(deg_range[0], deg_range[1] + 1, size=n_curves)
    ncps = rng.integers(ncp_range[0], ncp_range[1] + 1, size=n_curves)
    knots, cps = [], []
    for p, ncp in zip(degs, ncps):
        p, ncp = int(p), int(ncp)
        knots.append(random_clamped_knots(rng, p, ncp))
        cps.append(rng.uniform(0.0, 1.0, size=(ncp, 3)))
    cs = pack_curves(degs, knots, cps)
    lo, hi = cp_boxes(cs)
    pc = rng.integers(0, n_curves, size=n_proj).astype(np.int32)
    q = _box_queries(rng, lo, hi, pc)
    ic = rng.integers(0, n_curves, size=n_inv).astype(np.int32)
    t = rng.uniform(0.0, 1.0, size=n_inv)
    return cs, CurveQueries(pc, q, ic, t)


def nurbs_curve_set(seed: int = 4, n_curves: int = 4096, n_proj: int = 1_000_000, n_inv: int = 1_000_000,
                    deg_range=(2, 7), ncp_range=(8, 64), w_range=(0.5, 2.0)):
    """The ``curve_set`` recipe (degree ~U{2..7}, 8..64 control points
    ~U[0,1]^3, clamped non-uniform knots) with a weight per control point,
    log-uniform in w_range: rational curves (NURBS)."""
    rng = np.random.default_rng(seed)
    degs = rng.integers(deg_range[0], deg_range[1] + 1, size=n_curves)
    ncps = rng.integers(ncp_range[0], ncp_range[1] + 1, size=n_curves)
    knots, cps, ws = [], [], []
    lw0, lw1 = np.log(w_range[0]), np.log(w_range[1])
    for p, ncp in zip(degs, ncps):
        p, ncp = int(p), int(ncp)
        knots.append(random_clamped_knots(rng, p, ncp))
        cps.append(rng.uniform(0.0, 1.0, size=(ncp, 3)))
        ws.append(np.exp(rng.uniform(lw0, lw1, size=ncp)))
    cs = pack_curves(degs, knots, cps, ws)
    lo, hi = cp_boxes(cs)
    pc = rng.integers(0, n_curves, size=n_proj).astype(np.int32)
    q = _box_queries(rng, lo, hi, pc)
    ic = rng.integers(0, n_curves, size=n_inv).astype(np.int32)
    t = rng.uniform(0.0, 1.0, size=n_inv)
    return cs, CurveQueries(pc, q, ic, t)


def nurbs_circles(seed: int = 6, n_curves: int = 16, n_proj: int = 10_000):
    """Full circles as rational quadratic B-splines: nine control points on
    the square circumscribing the circle (corners carry weight sqrt(2)/2,
    the rest 1), knots 0,0,0,1/4,1/4,1/2,1/2,3/4,3/4,1,1,1.  Random centre
    ~U[0,1]^3, radius ~U[0.05,0.5] and plane (orthonormal e1, e2).
    Returns (cs, queries, centre [n][3], radius [n], normal [n][3]) so that
    a test can compare against the closed-form distance to a circle;
    queries ~U over the circle's box inflated 50% in every direction."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(0.5)
    unit = np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1], [1, 0]], np.float64)
    wts = np.array([1, s, 1, s, 1, s, 1, s, 1], np.float64)
    U = np.array([0, 0, 0, 0.25, 0.25, 0.5, 0.5, 0.75, 0.75, 1, 1, 1], np.float64)
    centre = rng.uniform(0.0, 1.0, size=(n_curves, 3))
    radius = rng.uniform(0.05, 0.5, size=n_curves)
    normal = np.zeros((n_curves, 3))
    cps = []
    for c in range(n_curves):
        a = rng.normal(size=3)
        e1 = a / np.linalg.norm(a)
        b = rng.normal(size=3)
        b -= (b @ e1) * e1
        e2 = b / np.linalg.norm(b)
        normal[c] = np.cross(e1, e2)
        cps.append(centre[c] + radius[c] * (unit[:, :1] * e1 + unit[:, 1:] * e2))
    cs = pack_curves([2] * n_curves, [U] * n_curves, cps, [wts] * n_curves)
    pc = rng.integers(0, n_curves, size=n_proj).astype(np.int32)
    q = centre[pc] + 1.5 * radius[pc, None] * rng.uniform(-1.0, 1.0, size=(n_proj, 3))
    return cs, CurveQueries(pc, q, np.zeros(0, np.int32), np.zeros(0)), centre, radius, normal


# The paper's 18 test curves (its per-module tables for the 2D models a-i
# and the 3D models j-r): (model, dimension, degree, knot-vector length,
# control points).  The curves themselves are not published: these shapes
# with random control points stand in for them.
PAPER_MODELS = (
    ("a", 2, 4, 10, 5), ("b", 2, 5, 12, 6), ("c", 2, 6, 14, 7), ("d", 2, 4, 14, 9), ("e", 2, 5, 18, 12),
    ("f", 2, 6, 22, 15), ("g", 2, 4, 35, 30), ("h", 2, 5, 22, 16), ("i", 2, 6, 57, 50),
    ("j", 3, 4, 10, 5), ("k", 3, 5, 12, 6), ("l", 3, 6, 14, 7), ("m", 3, 4, 14, 9), ("n", 3, 5, 18, 12),
    ("o", 3, 6, 22, 15), ("p", 3, 4, 35, 30), ("q", 3, 5, 46, 40), ("r", 3, 6, 57, 50),
)


def paper_suite(seed: int = 17, n_proj: int = 10_000, n_inv: int = 10_000):
    """One curve per paper model (curve index = position in PAPER_MODELS):
    the model's degree and control-point count, uniform clamped knots,
    control points ~U[0,1]^2 with z = 0 for the 2D models and ~U[0,1]^3 for
    the 3D ones; per model n_proj projection queries ~U over its control-
    point box inflated 20% (z = 0 for 2D) and n_inv inversion parameters
    ~U[0,1].  Queries are grouped by model."""
    rng = np.random.default_rng(seed)
    degs, knots, cps = [], [], []
    for _, dim, p, klen, ncp in PAPER_MODELS:
        assert klen == ncp + p + 1
        P = np.zeros((ncp, 3))
        P[:, :dim] = rng.uniform(0.0, 1.0, size=(ncp, dim))
        degs.append(p)
        knots.append(uniform_clamped_knots(p, ncp))
        cps.append(P)
    cs = pack_curves(degs, knots, cps)
    lo, hi = cp_boxes(cs)
    n = len(PAPER_MODELS)
    pc = np.repeat(np.arange(n, dtype=np.int32), n_proj)
    q = _box_queries(rng, lo, hi, pc)
    ic = np.repeat(np.arange(n, dtype=np.int32), n_inv)
    t = rng.uniform(0.0, 1.0, size=n * n_inv)
    return cs, CurveQueries(pc, q, ic, t)


# --------------------------------------------------------------------------
# surface workloads
# --------------------------------------------------------------------------

@dataclass
class SurfaceQueries:
    """Projection queries: surface id, (u,v) of a base point, direction w on
    the unit sphere and radius r (the point is S(u,v) + r w, formed by the
    caller).  Inversion queries: surface id and (u,v)."""

    proj_surf: np.ndarray
    proj_uv: np.ndarray
    proj_dir: np.ndarray
    proj_r: np.ndarray
    inv_surf: np.ndarray
    inv_uv: np.ndarray


def _sinusoid_net(rng, nu, nv):
    x = np.arange(nu, dtype=np.float64) / (nu - 1)
    y = np.arange(nv, dtype=np.float64) / (nv - 1)
    X, Y = np.meshgrid(x, y, indexing="ij")
    Z = np.zeros_like(X)
    for _ in range(3):
        a = rng.uniform(0.05, 0.3)
        f = rng.uniform(0.5, 3.0)
        th = rng.uniform(0.0, 2 * np.pi)
        ph = rng.uniform(0.0, 2 * np.pi)
        Z += a * np.sin(2 * np.pi * f * (np.cos(th) * X + np.sin(th) * Y) + ph)
    Z += rng.normal(0.0, 0.05, size=Z.shape)
    return np.stack([X, Y, Z], axis=-1)


def sphere_dirs(rng, n):
    w = rng.normal(size=(n, 3))
    return w / np.linalg.norm(w, axis=1, keepdims=True)


def surface_set(seed: int = 3, n_surf: int = 1024, n_proj: int = 4_000_000, n_inv: int = 4_000_000,
                deg_range=(2, 5), n_range=(8, 32), radius_frac: float = 0.2):
    """Random surfaces: bi-degree ~U{2..5}^2, nets n_u,n_v ~U{8..32} on a
    regular grid in [0,1]^2 with z = sum of 3 random sinusoids + N(0,0.05^2)
    noise, clamped non-uniform knots as for curve_set."""
    rng = np.random.default_rng(seed)
    pus = rng.integers(deg_range[0], deg_range[1] + 1, size=n_surf)
    pvs = rng.integers(deg_range[0], deg_range[1] + 1, size=n_surf)
    nus = rng.integers(n_range[0], n_range[1] + 1, size=n_surf)
    nvs = rng.integers(n_range[0], n_range[1] + 1, size=n_surf)
    KU, KV, nets = [], [], []
    for pu, pv, nu, nv in zip(pus, pvs, nus, nvs):
        KU.append(random_clamped_knots(rng, int(pu), int(nu)))
        KV.append(random_clamped_knots(rng, int(pv), int(nv)))
        nets.append(_sinusoid_net(rng, int(nu), int(nv)))
    ss = pack_surfaces(pus, pvs, KU, KV, nets)
    lo = np.minimum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    hi = np.maximum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    diag = np.linalg.norm(hi - lo, axis=1)
    ps = rng.integers(0, n_surf, size=n_proj).astype(np.int32)
    puv = rng.uniform(0.0, 1.0, size=(n_proj, 2))
    pdir = sphere_dirs(rng, n_proj)
    pr = rng.uniform(0.0, radius_frac, size=n_proj) * diag[ps]
    isf = rng.integers(0, n_surf, size=n_inv).astype(np.int32)
    iuv = rng.uniform(0.0, 1.0, size=(n_inv, 2))
    return ss, SurfaceQueries(ps, puv, pdir, pr, isf, iuv)


# --------------------------------------------------------------------------
# ragged mixed batch
# --------------------------------------------------------------------------

def lognormal_counts(rng, n, mu=np.log(48.0), sigma=1.3, lo=1, hi=2000):
    return np.clip(np.round(rng.lognormal(mu, sigma, size=n)), lo, hi).astype(np.int64)


def zipf_assign(rng, n_items, n_queries, s=1.1):
    """Query -> item assignment with Zipf(s) weights over a random rank permutation."""
    ranks = np.arange(1, n_items + 1, dtype=np.float64)
    w = ranks ** (-s)
    w /= w.sum()
    perm = rng.permutation(n_items)
    return perm[rng.choice(n_items, size=n_queries, p=w)].astype(np.int32)


def ragged_mix(seed: int = 5, n_curves: int = 65_536, n_surf: int = 8_192, n_queries: int = 64_000_000):
    """Cubic curves with n+3 control points (n segments) and bicubic surfaces
    with n_u*n_v ~ n patches, n ~ round(LogNormal(ln 48, 1.3)) in [1, 2000];
    queries split half projection / half inversion, Zipf(1.1)-skewed."""
    rng = np.random.default_rng(seed)
    nc = lognormal_counts(rng, n_curves)
    knots, cps = [], []
    for n in nc:
        ncp = int(n) + 3
        knots.append(uniform_clamped_knots(3, ncp))
        cps.append(np.cumsum(rng.uniform(-0.1, 0.1, size=(ncp, 3)), axis=0) + rng.uniform(0, 1, size=3))
    cs = pack_curves(np.full(n_curves, 3), knots, cps)
    ns = lognormal_counts(rng, n_surf)
    KU, KV, nets = [], [], []
    for n in ns:
        a = max(1, int(round(np.sqrt(float(n)))))
        b = max(1, int(round(float(n) / a)))
        nu, nv = a + 3, b + 3
        KU.append(uniform_clamped_knots(3, nu))
        KV.append(uniform_clamped_knots(3, nv))
        nets.append(_sinusoid_net(rng, nu, nv))
    ss = pack_surfaces(np.full(n_surf, 3), np.full(n_surf, 3), KU, KV, nets)
    half = n_queries // 2
    qc = zipf_assign(rng, n_curves, half)
    qs = zipf_assign(rng, n_surf, n_queries - half)
    return cs, ss, qc, qs, rng


def ragged_queries(cs: CurveSet, ss: SurfaceSet, qc, qs, rng, radius_frac: float = 0.2):
    """Query recipes of the ragged batch: the first half of each spline kind's
    queries are projections, the rest inversions.  Curves: points uniform in
    the curve's control-point box scaled 1.2x, inversion parameters t ~ U[0,1];
    surfaces: S(u,v) + r w with (u,v) ~ U[0,1]^2, w on the unit sphere and
    r ~ U[0, radius_frac] x the surface's box diagonal, inversion (u,v) ~ U[0,1]^2."""
    hc, hs = len(qc) // 2, len(qs) // 2
    lo, hi = cp_boxes(cs)
    pc = np.ascontiguousarray(qc[:hc])
    cq = CurveQueries(pc, _box_queries(rng, lo, hi, pc), np.ascontiguousarray(qc[hc:]),
                      rng.uniform(0.0, 1.0, size=len(qc) - hc))
    slo = np.minimum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    shi = np.maximum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    diag = np.linalg.norm(shi - slo, axis=1)
    ps = np.ascontiguousarray(qs[:hs])
    sq = SurfaceQueries(ps, rng.uniform(0.0, 1.0, size=(hs, 2)), sphere_dirs(rng, hs),
                        rng.uniform(0.0, radius_frac, size=hs) * diag[ps], np.ascontiguousarray(qs[hs:]),
                        rng.uniform(0.0, 1.0, size=(len(qs) - hs, 2)))
    return cq, sq


# ------------------------------------------------------------ learned seed

MLP_SHAPES = (("W1", (128, 16)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 128)),
              ("b3", (128,)), ("w4", (128,)), ("b4", (1,)))
MLP_NPARAM = 35332


SMLP_NPARAM = 41604
SMLP_SHAPES = (("W1", (128, 64)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 128)),
               ("b3", (128,)), ("W4", (2, 128)), ("b4", (2,)))


def smlp_init(seed: int = 8) -> np.ndarray:
    """Initial parameter vector of the surface seed network (layout of
    include/bspl_mlp.h, BSPL_SMLP_*): weights ~ N(0, 2 / fan_in), biases 0,
    the weight columns of the 13 zero inputs 0."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(SMLP_NPARAM, np.float32)
    o = 0
    for name, shp in SMLP_SHAPES:
        n = int(np.prod(shp))
        if name[0] in "Ww":
            fan_in = 51 if name == "W1" else 128
            w = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
            if name == "W1":
                w[:, 51:] = 0.0
            theta[o:o + n] = w.reshape(-1)
        o += n
    return theta


def mlp_init(seed: int = 7) -> np.ndarray:
    """Initial parameter vector of the seed network (layout of
    include/bspl_mlp.h): weights ~ N(0, 2 / fan_in), biases 0, the weight
    column of the zero input 0."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(MLP_NPARAM, np.float32)
    o = 0
    for name, shp in MLP_SHAPES:
        n = int(np.prod(shp))
        if name[0] in "Ww":
            fan_in = 15 if name == "W1" else 128
            w = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
            if name == "W1":
                w[:, 15] = 0.0
            theta[o:o + n] = w.reshape(-1)
        o += n
    return theta


def nurbs_edge_set(seed: int = 7):
    """Rational edge cases: a degree-1 curve with unequal weights (a line
    with a non-uniform parameterisation), a quarter circle (degree 2, weights
    1, sqrt(2)/2, 1), a cubic with a C0 joint (interior knot of multiplicity
    3), a single degree-7 span, a cubic on the domain [-3, 5], and a quartic
    whose weights span 50:1.  Control points ~U[0,1]^3 where not fixed."""
    rng = np.random.default_rng(seed)
    degs, knots, cps, ws = [], [], [], []

    def add(p, U, P, w):
        degs.append(p)
        knots.append(np.asarray(U, np.float64))
        cps.append(np.asarray(P, np.float64))
        ws.append(np.asarray(w, np.float64))

    add(1, [0, 0, 1, 1], rng.uniform(0, 1, (2, 3)), [1.0, 3.0])
    add(2, [0, 0, 0, 1, 1, 1], [[1, 0, 0], [1, 1, 0], [0, 1, 0]], [1.0, np.sqrt(0.5), 1.0])
    add(3, [0, 0, 0, 0, 0.4, 0.4, 0.4, 0.7, 1, 1, 1, 1], rng.uniform(0, 1, (8, 3)),
        np.exp(rng.uniform(np.log(0.5), np.log(2.0), 8)))
    add(7, uniform_clamped_knots(7, 8), rng.uniform(0, 1, (8, 3)), np.exp(rng.uniform(np.log(0.5), np.log(2.0), 8)))
    add(3, np.concatenate([[-3.0] * 4, [-1.0, 2.0], [5.0] * 4]), rng.uniform(0, 1, (6, 3)),
        np.exp(rng.uniform(np.log(0.5), np.log(2.0), 6)))
    w = np.exp(rng.uniform(0.0, np.log(50.0), 10))
    w[0], w[-1] = 1.0, 50.0
    add(4, random_clamped_knots(rng, 4, 10), rng.uniform(0, 1, (10, 3)), w)
    return pack_curves(degs, knots, cps, ws)


def nurbs_surface_set(seed: int = 8, n_surf: int = 64, n_proj: int = 10_000, deg_range=(2, 5), n_range=(8, 16),
                      w_range=(0.5, 2.0)):
    """The surface_set recipe (sinusoid nets on a grid, clamped non-uniform
    knots) with one weight per control point, log-uniform in w_range:
    rational surfaces; projection queries as for surface_set."""
    ss, sq = surface_set(seed=seed, n_surf=n_surf, n_proj=n_proj, n_inv=0, deg_range=deg_range, n_range=n_range)
    rng = np.random.default_rng(seed + 1)
    ss.weights = np.exp(rng.uniform(np.log(w_range[0]), np.log(w_range[1]), size=len(ss.cps)))
    return ss, sq


def nurbs_cylinders(seed: int = 9, n_surf: int = 8, n_proj: int = 2000):
    """Open cylinders as rational surfaces: along u the full circle of
    nurbs_circles (degree 2, nine control points, corner weights
    sqrt(2)/2), along v a straight segment (degree 1) of height h along the
    axis.  Random centre ~U[0,1]^3, radius ~U[0.05, 0.5], height
    ~U[0.2, 1], axis direction.  Returns (ss, queries [n][3], surface index
    [n], centre [n_surf][3], axis [n_surf][3], radius, height); queries lie
    at heights ~U[0.1 h, 0.9 h] and radial distances ~U[0, 2 r] from the
    axis, so that the nearest point is on the cylinder's side."""
    rng = np.random.default_rng(seed)
    s2 = np.sqrt(0.5)
    unit = np.array([[1, 0], [1, 1], [0, 1], [-1, 1], [-1, 0], [-1, -1], [0, -1], [1, -1], [1, 0]], np.float64)
    wc = np.array([1, s2, 1, s2, 1, s2, 1, s2, 1], np.float64)
    U = np.array([0, 0, 0, 0.25, 0.25, 0.5, 0.5, 0.75, 0.75, 1, 1, 1], np.float64)
    V = np.array([0, 0, 1, 1], np.float64)
    centre = rng.uniform(0.0, 1.0, size=(n_surf, 3))
    radius = rng.uniform(0.05, 0.5, size=n_surf)
    height = rng.uniform(0.2, 1.0, size=n_surf)
    axis = np.zeros((n_surf, 3))
    nets, ws, frames = [], [], []
    for c in range(n_surf):
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        e1 = rng.normal(size=3)
        e1 -= (e1 @ a) * a
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(a, e1)
        axis[c] = a
        ring = centre[c] + radius[c] * (unit[:, :1] * e1 + unit[:, 1:] * e2)   # [9][3]
        nets.append(np.stack([ring, ring + height[c] * a], axis=1))            # [9][2][3]
        ws.append(np.stack([wc, wc], axis=1))
        frames.append((e1, e2))
    ss = pack_surfaces([2] * n_surf, [1] * n_surf, [U] * n_surf, [V] * n_surf, nets, ws)
    sidx = rng.integers(0, n_surf, size=n_proj).astype(np.int32)
    hq = rng.uniform(0.1, 0.9, size=n_proj) * height[sidx]
    rq = rng.uniform(0.0, 2.0, size=n_proj) * radius[sidx]
    ang = rng.uniform(0.0, 2 * np.pi, size=n_proj)
    e1 = np.array([frames[c][0] for c in sidx])
    e2 = np.array([frames[c][1] for c in sidx])
    q = centre[sidx] + hq[:, None] * axis[sidx] + rq[:, None] * (np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2)
    return ss, q, sidx, centre, axis, radius, height
