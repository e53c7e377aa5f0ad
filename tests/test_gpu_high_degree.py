"""Curves of degree 32..63 (above the paper's limit of 31) on the GPU,
through the C ABI, against the oracle: decomposition bit-exact (each span
extracted from the blossom), evaluation, projection refined on the original
curve and inversion, for non-rational and rational curves."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def high_set(rational):
    rng = np.random.default_rng(52)
    degs, knots, cps, ws = [], [], [], []
    for p in (3, 31, 32, 40, 51, 63):
        ncp = p + int(rng.integers(1, 8))
        degs.append(p)
        knots.append(synth.random_clamped_knots(rng, p, ncp))
        cps.append(rng.uniform(0.0, 1.0, size=(ncp, 3)))
        ws.append(np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncp)))
    return synth.pack_curves(degs, knots, cps, ws if rational else None)


@pytest.mark.parametrize("rational", [False, True])
def test_high_degree_curves_vs_oracle(rational):
    cs = high_set(rational)
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    ref = O.decompose_curves(cs, TOL)
    n = ref.total
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)
    assert np.array_equal(segs.ctrl[:n].cpu().numpy().reshape(n, 4, 3), ref.ctrl)
    assert np.array_equal(segs.prange[:n].cpu().numpy().reshape(n, 2), ref.prange)
    rng = np.random.default_rng(53)
    t = rng.uniform(0.0, 1.0, 3000)
    qc_e = np.repeat(np.arange(cs.n, dtype=np.int32), 500)
    got = bspl.bspl_eval_curves(dc, dev(qc_e, torch.int32), dev(t, torch.float64)).cpu().numpy()
    assert np.abs(got - O.eval_curves(cs, qc_e, t)[0]).max() <= 1e-13
    lo, hi = synth.cp_boxes(cs)
    q_h = synth._box_queries(rng, lo, hi, qc_e, scale=1.3)
    _, d_o = O.project_curves(cs, qc_e, q_h)
    diag = O.curve_diag(cs)[qc_e]
    qc, q = dev(qc_e, torch.int32), dev(q_h, torch.float64)
    for prec in (bspl.FP64, bspl.MIXED, bspl.LEARNED_MIXED):
        r = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=prec))
        bspl.bspl_refine_curves(dc, qc, q, r, ws=bspl.refine_workspace(dc, len(qc_e), DEV))
        torch.cuda.synchronize()
        err = np.abs(r.dist.cpu().numpy() - d_o) / diag
        assert err.max() <= 1e-9, (prec, int((err > 1e-9).sum()), err.max())
    pts = bspl.bspl_eval_curves(dc, qc, dev(t, torch.float64))
    ri = bspl.bspl_invert_curves(segs, qc, pts, bspl.make_options(prec=bspl.MIXED))
    bspl.bspl_refine_curves(dc, qc, pts, ri, invert=True, diag=segs.diag)
    torch.cuda.synchronize()
    assert np.all(ri.dist.cpu().numpy() <= 1e-9 * diag)
