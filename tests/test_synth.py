"""Input recipes of the ragged batch (CPU): shapes, the projection /
inversion split, log-normal piece counts, Zipf skew and query ranges."""
import numpy as np

from paper_2504_11498_gb300 import synth


def test_ragged_batch_recipe():
    cs, ss, qc, qs, rng = synth.ragged_mix(seed=5, n_curves=4096, n_surf=512, n_queries=200_000)
    assert cs.n == 4096 and ss.n == 512 and len(qc) == len(qs) == 100_000
    assert np.all(cs.degree == 3) and np.all(ss.deg_u == 3) and np.all(ss.deg_v == 3)
    n_seg = np.diff(cs.cp_off) - 3
    assert n_seg.min() >= 1 and n_seg.max() <= 2000
    # log-normal(ln 48, 1.3): the median piece count is near 48
    assert 40 <= np.median(n_seg) <= 56
    # Zipf(1.1): the most popular curve draws far more than the uniform share
    assert np.bincount(qc, minlength=cs.n).max() > 50 * len(qc) / cs.n
    cq, sq = synth.ragged_queries(cs, ss, qc, qs, rng)
    assert len(cq.proj_curve) == len(cq.inv_curve) == 50_000
    assert len(sq.proj_surf) == len(sq.inv_surf) == 50_000
    assert np.array_equal(np.concatenate([cq.proj_curve, cq.inv_curve]), qc)
    assert np.array_equal(np.concatenate([sq.proj_surf, sq.inv_surf]), qs)
    lo, hi = synth.cp_boxes(cs)
    c, h = 0.5 * (lo + hi), 0.6 * (hi - lo)
    k = cq.proj_curve
    assert np.all(np.abs(cq.proj_xyz - c[k]) <= h[k] + 1e-12)
    assert np.all((cq.inv_t >= 0) & (cq.inv_t <= 1))
    assert np.all((sq.proj_uv >= 0) & (sq.proj_uv <= 1)) and np.all((sq.inv_uv >= 0) & (sq.inv_uv <= 1))
    assert np.allclose(np.linalg.norm(sq.proj_dir, axis=1), 1.0)
    slo = np.minimum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    shi = np.maximum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    diag = np.linalg.norm(shi - slo, axis=1)
    assert np.all((sq.proj_r >= 0) & (sq.proj_r <= 0.2 * diag[sq.proj_surf]))


def test_paper_suite_recipe():
    """One curve per paper model with its degree, knot-vector length and
    control-point count; 2D models (a-i) at z = 0; uniform clamped knots on
    [0, 1]; queries grouped by model inside the inflated control box."""
    cs, cq = synth.paper_suite(seed=17, n_proj=1000, n_inv=500)
    assert cs.n == 18
    for c, (name, dim, p, klen, ncp) in enumerate(synth.PAPER_MODELS):
        deg, U, P = cs.curve(c)
        assert (deg, len(U), len(P)) == (p, klen, ncp)
        assert np.all(U[:p + 1] == 0) and np.all(U[-p - 1:] == 1)
        assert np.allclose(np.diff(U[p:len(U) - p]), 1.0 / (ncp - p))
        assert np.all((P[:, :dim] >= 0) & (P[:, :dim] <= 1))
        if dim == 2:
            assert np.all(P[:, 2] == 0) and np.all(cq.proj_xyz[cq.proj_curve == c, 2] == 0)
    assert np.array_equal(cq.proj_curve, np.repeat(np.arange(18), 1000))
    assert np.array_equal(cq.inv_curve, np.repeat(np.arange(18), 500))
    lo, hi = synth.cp_boxes(cs)
    c, h = 0.5 * (lo + hi), 0.6 * (hi - lo)
    k = cq.proj_curve
    assert np.all(np.abs(cq.proj_xyz - c[k]) <= h[k] + 1e-12)


def test_nurbs_recipes():
    """The NURBS set: the curve-set recipe plus one weight per control point,
    log-uniform in [1/2, 2]; circles: nine control points on the square
    around the circle in its plane, corner weights sqrt(2)/2; the edge set's
    curves; weights carried through subset()."""
    cs, qs = synth.nurbs_curve_set(seed=4, n_curves=512, n_proj=1000, n_inv=500)
    assert cs.weights.shape == (len(cs.cps),)
    lw = np.log(cs.weights)
    assert lw.min() >= np.log(0.5) and lw.max() <= np.log(2.0)
    # log-uniform: mean of log w near 0, spread near (ln 4)/sqrt(12)
    assert abs(lw.mean()) < 0.02 and abs(lw.std() - np.log(4.0) / np.sqrt(12.0)) < 0.02
    assert np.all((cs.degree >= 2) & (cs.degree <= 7))
    sub = cs.subset([3, 1])
    assert np.array_equal(sub.weights, np.concatenate([cs.curve_weights(3), cs.curve_weights(1)]))
    circ, cq, centre, radius, normal = synth.nurbs_circles(seed=6, n_curves=5, n_proj=100)
    assert np.all(circ.degree == 2) and circ.weights.shape == (45,)
    for c in range(circ.n):
        _, U, P = circ.curve(c)
        w = circ.curve_weights(c)
        assert np.allclose(w[1::2], np.sqrt(0.5)) and np.all(w[0::2] == 1.0)
        d = P - centre[c]
        assert np.allclose(d @ normal[c], 0.0, atol=1e-14)
        # edge midpoints at the radius, corners at radius * sqrt(2)
        r = np.linalg.norm(d, axis=1)
        assert np.allclose(r[0::2], radius[c]) and np.allclose(r[1::2], radius[c] * np.sqrt(2.0))
        assert np.array_equal(U, [0, 0, 0, .25, .25, .5, .5, .75, .75, 1, 1, 1])
    edge = synth.nurbs_edge_set()
    assert edge.n == 6 and list(edge.degree) == [1, 2, 3, 7, 3, 4]
    assert edge.curve_weights(5).max() / edge.curve_weights(5).min() == 50.0
    p, U, _ = edge.curve(4)
    assert U[p] == -3.0 and U[-1] == 5.0


def test_refine_flop_count():
    """The refinement's counted flops per evaluation of degree p (the
    benchmark's roofline numerator)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ev = [0] * 64
    ev[3] = 10     # full evaluations of a cubic: 18 + 12 + 72 + 27 + 30 = 159 each
    ev[32 + 3] = 5  # C and C' alone: 18 + 12 + 56 + 14 + 30 = 130 each
    assert bench.refine_flops(ev) == 10 * 159 + 5 * 130
    # non-rational: 3 coordinates, no quotient
    assert bench.refine_flops(ev, rational=False) == 10 * (18 + 12 + 54 + 30) + 5 * (18 + 12 + 42 + 30)
