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


def test_refine_reaches_minima_at_c0_joints():
    """Starts 1e-9 and 1e-6 either side of minima on or next to the C0 joint
    of the cubic in the set above: the refinement (through the C ABI) ends
    within 1e-9 x diag of the oracle (the full step from the far side of the
    joint is first replaced by the knot it crossed)."""
    cs = high_set(False)
    p, U, P = cs.curve(0)
    inner, counts = np.unique(U[p + 1:len(P)], return_counts=True)
    joints = inner[counts >= p]
    assert len(joints) >= 1
    rng = np.random.default_rng(53)
    rng.uniform(0.0, 1.0, 3000)
    qc_all = np.repeat(np.arange(cs.n, dtype=np.int32), 500)
    lo, hi = synth.cp_boxes(cs)
    q_all = synth._box_queries(rng, lo, hi, qc_all, scale=1.3)
    sel = np.where(qc_all == 0)[0]
    t_o, d_o = O.project_curves(cs, qc_all[sel], q_all[sel])
    near = np.where(np.min(np.abs(t_o[:, None] - joints[None, :]), axis=1) <= 1e-5)[0]
    assert len(near) >= 5
    offs = np.array([-1e-6, -1e-9, 1e-9, 1e-6])
    t0 = np.clip(np.repeat(t_o[near], 4) + np.tile(offs, len(near)), U[p], U[len(P)])
    q = np.repeat(q_all[sel][near], 4, axis=0)
    dc = bspl.DeviceCurves(cs, DEV)
    qc = dev(np.zeros(len(t0), np.int32), torch.int32)
    r = bspl.QueryResult(dev(t0, torch.float64), dev(np.zeros(len(t0)), torch.float64),
                         dev(np.zeros(len(t0), np.uint8), torch.uint8))
    bspl.bspl_refine_curves(dc, qc, dev(q, torch.float64), r)
    torch.cuda.synchronize()
    err = np.abs(r.dist.cpu().numpy() - np.repeat(d_o[near], 4)) / O.curve_diag(cs)[0]
    assert err.max() <= 1e-9, (int((err > 1e-9).sum()), err.max())
