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
