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
