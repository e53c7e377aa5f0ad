"""GPU parity of the rational-curve (NURBS) path, through the C ABI, against
the CPU oracle.

* decomposition (homogeneous span pieces, Hermite cubics, certified bound):
  offsets, control points and parameter ranges bit-exact;
* evaluation of the original rational curves;
* projection and inversion: every query path on the decomposed curves, then
  rational Newton on the original curves (bspl_refine_curves).  Before the
  refinement the distance is the cubic approximant's, within tol x diag of
  the oracle's; after it the distance is the original curve's, within
  1e-9 x diag of the oracle's on every query;
* exact circles against the closed-form distance;
* equal weights give the non-rational results; invalid weights -> EINVAL.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def small_set(n=96, seed=41, n_proj=20_000, n_inv=5_000, w_range=(0.5, 2.0)):
    return synth.nurbs_curve_set(seed=seed, n_curves=n, n_proj=n_proj, n_inv=n_inv, w_range=w_range)


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-10])
def test_nurbs_decompose_bit_exact(tol):
    cs, _ = small_set(w_range=(0.25, 4.0))
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), tol)
    ref = O.decompose_curves(cs, tol)
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)
    n = ref.total
    assert np.array_equal(segs.ctrl[:n].cpu().numpy().reshape(n, 4, 3), ref.ctrl)
    assert np.array_equal(segs.prange[:n].cpu().numpy().reshape(n, 2), ref.prange)


def test_nurbs_full_set_counts():
    """The 4,096-curve NURBS set at the benchmark's tolerance: segment
    counts bit-exact with the oracle."""
    cs, _ = synth.nurbs_curve_set(seed=4, n_proj=0, n_inv=0)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), TOL)
    ref = O.decompose_curves(cs, TOL, count_only=True)
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)


def test_nurbs_eval():
    cs, qs = small_set()
    dc = bspl.DeviceCurves(cs, DEV)
    rng = np.random.default_rng(3)
    qc = rng.integers(0, cs.n, 50_000).astype(np.int32)
    t = rng.uniform(-0.05, 1.05, 50_000)  # clamped outside the domain
    got = bspl.bspl_eval_curves(dc, dev(qc, torch.int32), dev(t, torch.float64)).cpu().numpy()
    ref = O.eval_curves(cs, qc, np.clip(t, 0.0, 1.0))[0]
    assert np.abs(got - ref).max() <= 1e-14


def _paths():
    return [bspl.FP64, bspl.MIXED, bspl.LEARNED_MIXED, bspl.CLIP_MIXED]


@pytest.mark.parametrize("prec", _paths())
def test_nurbs_projection_and_inversion_refined_vs_oracle(prec):
    cs, qs = small_set()
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    diag_all = O.curve_diag(cs)
    mlp = bspl.Mlp(synth.mlp_init(21)) if prec == bspl.LEARNED_MIXED else None
    o = bspl.make_options(prec=prec, mlp=mlp)
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    r = bspl.bspl_project_curves(segs, qc, q, o)
    torch.cuda.synchronize()
    d_apx = r.dist.cpu().numpy().copy()
    t_o, d_o = O.project_curves(cs, qs.proj_curve, qs.proj_xyz)
    diag = diag_all[qs.proj_curve]
    assert np.all(np.abs(d_apx - d_o) <= TOL * diag + 1e-12 * diag)
    bspl.bspl_refine_curves(dc, qc, q, r)
    torch.cuda.synchronize()
    t_r, d_r, s_r = (x.cpu().numpy().copy() for x in (r.param, r.dist, r.status))
    err = np.abs(d_r - d_o) / diag
    assert err.max() <= 1e-9, (prec, int((err > 1e-9).sum()), err.max())
    # the refined distance is the original curve's at the refined parameter
    C = O.eval_curves(cs, qs.proj_curve, t_r)[0]
    assert np.abs(np.linalg.norm(C - qs.proj_xyz, axis=1) - d_r).max() <= 1e-13
    assert not np.any(s_r & bspl.Q_INVALID)
    # inversion: points on the original curve
    ic = dev(qs.inv_curve, torch.int32)
    pts = bspl.bspl_eval_curves(dc, ic, dev(qs.inv_t, torch.float64))
    ri = bspl.bspl_invert_curves(segs, ic, pts, o)
    bspl.bspl_refine_curves(dc, ic, pts, ri, invert=True, diag=segs.diag)
    torch.cuda.synchronize()
    di, si = ri.dist.cpu().numpy(), ri.status.cpu().numpy()
    dgi = diag_all[qs.inv_curve]
    assert np.all(di <= 1e-9 * dgi), np.max(di / dgi)
    assert not np.any(si & bspl.Q_OFF_CURVE)


def test_nurbs_circles_closed_form():
    cs, qs, centre, radius, normal = synth.nurbs_circles(n_curves=64, n_proj=100_000)
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    c = qs.proj_curve
    v = qs.proj_xyz - centre[c]
    h = np.einsum("ij,ij->i", v, normal[c])
    rho = np.linalg.norm(v - h[:, None] * normal[c], axis=1)
    exact = np.sqrt(h * h + (rho - radius[c]) ** 2)
    for prec in (bspl.MIXED, bspl.LEARNED_MIXED):
        r = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=prec))
        bspl.bspl_refine_curves(dc, qc, q, r)
        torch.cuda.synchronize()
        d = r.dist.cpu().numpy()
        assert np.abs(d - exact).max() <= 1e-12 * radius.max(), (prec, np.abs(d - exact).max())


def test_nurbs_equal_weights_match_non_rational():
    cs, qs = synth.curve_set(seed=9, n_curves=64, n_proj=20_000, n_inv=0)
    rat = synth.CurveSet(cs.degree, cs.knot_off, cs.knots, cs.cp_off, cs.cps, np.full(len(cs.cps), 2.5))
    d0, d1 = bspl.DeviceCurves(cs, DEV), bspl.DeviceCurves(rat, DEV)
    s0, s1 = bspl.decompose(d0, TOL), bspl.decompose(d1, TOL)
    n = int(s0.seg_off[-1])
    assert torch.equal(s0.seg_off, s1.seg_off) and torch.equal(s0.ctrl[:n], s1.ctrl[:n])
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    o = bspl.make_options(prec=bspl.MIXED)
    r0 = bspl.bspl_refine_curves(d0, qc, q, bspl.bspl_project_curves(s0, qc, q, o))
    r1 = bspl.bspl_refine_curves(d1, qc, q, bspl.bspl_project_curves(s1, qc, q, o))
    torch.cuda.synchronize()
    assert torch.allclose(r0.dist, r1.dist, rtol=0, atol=1e-13)


def test_nurbs_invalid_weights():
    cs, _ = small_set(n=8, n_proj=0, n_inv=0)
    for bad in (0.0, -0.5, float("nan"), float("inf")):
        w = cs.weights.copy()
        w[7] = bad
        bad_cs = synth.CurveSet(cs.degree, cs.knot_off, cs.knots, cs.cp_off, cs.cps, w)
        with pytest.raises(bspl.BsplError):
            bspl.decompose(bspl.DeviceCurves(bad_cs, DEV), 1e-6)


def test_nurbs_full_size_sampled_parity():
    """The NURBS workload at the size the benchmark times (4,096 curves, 1M
    projection queries, learned path + refinement, as one graph replay):
    against the plain path + refinement on every query, against the oracle
    on a 30k sample."""
    cs, qs = synth.nurbs_curve_set(seed=4, n_proj=1_000_000, n_inv=0)
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    mlp = bspl.Mlp(synth.mlp_init(21))
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    buf = bspl.QueryBuffers(segs, len(qs.proj_curve), DEV, learned=True)
    o = bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp)
    rws = bspl.refine_workspace(dc, len(qs.proj_curve), DEV)

    def step():
        r = bspl.bspl_project_curves(segs, qc, q, o, buf)
        bspl.bspl_refine_curves(dc, qc, q, r, ws=rws)

    step()
    torch.cuda.synchronize()
    with bspl.Graph() as g:
        step()
    buf.dist.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    d_f, t_f = buf.dist.cpu().numpy().copy(), buf.param.cpu().numpy().copy()
    plain = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=bspl.FP64))
    bspl.bspl_refine_curves(dc, qc, q, plain)
    torch.cuda.synchronize()
    d_p = plain.dist.cpu().numpy()
    diag = O.curve_diag(cs)[qs.proj_curve]
    rel = np.abs(d_f - d_p) / diag
    assert np.all(np.isfinite(d_f)) and rel.max() <= 1e-9, (int((rel > 1e-9).sum()), rel.max())
    pick = np.random.default_rng(5).choice(len(d_f), 30_000, replace=False)
    _, d_o = O.project_curves(cs, qs.proj_curve[pick], qs.proj_xyz[pick])
    err = np.abs(d_f[pick] - d_o) / diag[pick]
    assert err.max() <= 1e-9, (int((err > 1e-9).sum()), err.max())
    assert bspl.mlp_check() == bspl.OK


def test_refine_grouped_by_curve_matches_caller_order():
    """The refinement with a workspace (queries grouped by curve, the
    per-span factors computed once per call) gives the same results, bit for
    bit, and the same evaluation counts as in the caller's order without
    one, and so does a workspace with room for only some curves' factors; a
    workspace below the grouping's size is refused."""
    cs, qs = small_set(n=64, n_proj=30_000, n_inv=0)
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    r = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=bspl.MIXED))
    a = bspl.QueryResult(r.param.clone(), r.dist.clone(), r.status.clone())
    ea = torch.zeros(bspl.REFINE_EVALS, dtype=torch.int64, device=DEV)
    eb = torch.zeros_like(ea)
    bspl.bspl_refine_curves(dc, qc, q, a, evals=ea)
    ws = bspl.refine_workspace(dc, len(qs.proj_curve), DEV)
    bspl.bspl_refine_curves(dc, qc, q, r, evals=eb, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(a.param, r.param) and torch.equal(a.dist, r.dist) and torch.equal(a.status, r.status)
    assert torch.equal(ea, eb) and int(ea.sum()) >= len(qs.proj_curve)
    # a workspace holding the grouping and the factors of only some curves
    part = bspl.workspace_bytes(bspl.OP_REFINE_CURVES, dc.n, dc.n_cp_total // 3, 0, len(qs.proj_curve))
    r2 = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=bspl.MIXED))
    bspl.bspl_refine_curves(dc, qc, q, r2, ws=ws[:part])
    torch.cuda.synchronize()
    assert torch.equal(a.param, r2.param) and torch.equal(a.dist, r2.dist) and torch.equal(a.status, r2.status)
    with pytest.raises(bspl.BsplError):
        bspl.bspl_refine_curves(dc, qc, q, r, ws=ws[:16])


@pytest.mark.parametrize("prec", _paths())
def test_nurbs_edge_curves(prec):
    """Rational edge cases (synth.nurbs_edge_set: a line with unequal
    weights, a quarter circle, a C0 joint, one degree-7 span, the domain
    [-3, 5], weights over 50:1): decomposition bit-exact, projection and
    inversion refined against the oracle on every query."""
    cs = synth.nurbs_edge_set()
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, TOL)
    ref = O.decompose_curves(cs, TOL)
    n = ref.total
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)
    assert np.array_equal(segs.ctrl[:n].cpu().numpy().reshape(n, 4, 3), ref.ctrl)
    rng = np.random.default_rng(9)
    lo, hi = synth.cp_boxes(cs)
    qc_h = np.repeat(np.arange(cs.n, dtype=np.int32), 500)
    q_h = synth._box_queries(rng, lo, hi, qc_h, scale=1.5)
    _, d_o = O.project_curves(cs, qc_h, q_h)
    diag = O.curve_diag(cs)[qc_h]
    mlp = bspl.Mlp(synth.mlp_init(21)) if prec == bspl.LEARNED_MIXED else None
    o = bspl.make_options(prec=prec, mlp=mlp)
    qc, q = dev(qc_h, torch.int32), dev(q_h, torch.float64)
    r = bspl.bspl_project_curves(segs, qc, q, o)
    bspl.bspl_refine_curves(dc, qc, q, r, ws=bspl.refine_workspace(dc, len(qc_h), DEV))
    torch.cuda.synchronize()
    err = np.abs(r.dist.cpu().numpy() - d_o) / diag
    assert err.max() <= 1e-9, (prec, int((err > 1e-9).sum()), err.max())
    # inversion: parameters across each curve's own domain
    t_in = np.concatenate([np.linspace(cs.curve(c)[1][cs.curve(c)[0]], cs.curve(c)[1][len(cs.curve(c)[2])], 300)
                           for c in range(cs.n)])
    ic = dev(np.repeat(np.arange(cs.n, dtype=np.int32), 300), torch.int32)
    pts = bspl.bspl_eval_curves(dc, ic, dev(t_in, torch.float64))
    ri = bspl.bspl_invert_curves(segs, ic, pts, o)
    bspl.bspl_refine_curves(dc, ic, pts, ri, invert=True, diag=segs.diag)
    torch.cuda.synchronize()
    dgi = O.curve_diag(cs)[np.repeat(np.arange(cs.n), 300)]
    assert np.all(ri.dist.cpu().numpy() <= 1e-9 * dgi)
