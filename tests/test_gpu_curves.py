"""GPU parity of curve decomposition and curve projection/inversion, through
the C ABI, against the CPU oracle.

Decomposition: segment counts, offsets, control points and parameter ranges
bit-exact.  Queries: |d_gpu - d_oracle| <= tol x diag + 1e-12 x diag for
every query (the GPU reports the distance to the decomposed curve, which is
within tol x diag of the original everywhere), and the GPU parameter,
evaluated on the original curve by the oracle, is no worse than
d_oracle + 2 tol x diag + 1e-12 x diag.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def run_queries(segs, qc, q, invert=False, **kw):
    fn = bspl.bspl_invert_curves if invert else bspl.bspl_project_curves
    r = fn(segs, dev(qc, torch.int32), dev(q, torch.float64), bspl.make_options(**kw))
    torch.cuda.synchronize()
    return r.param.cpu().numpy().copy(), r.dist.cpu().numpy().copy(), r.status.cpu().numpy().copy()


def check_against_oracle(cs, qc, q, t_gpu, d_gpu, tol, extra=0.0):
    t_o, d_o = O.project_curves(cs, qc, q)
    diag = O.curve_diag(cs)[qc]
    bound = tol * diag + 1e-12 * diag + extra * diag
    err = np.abs(d_gpu - d_o)
    assert np.all(np.isfinite(d_gpu))
    bad = np.where(err > bound)[0]
    assert len(bad) == 0, (len(bad), err[bad][:5] / diag[bad][:5], qc[bad][:5])
    # the GPU parameter on the ORIGINAL curve
    C, _, _ = O.eval_curves(cs, qc, t_gpu)
    d_orig = np.linalg.norm(C - q, axis=1)
    assert np.all(d_orig <= d_o + 2 * tol * diag + 1e-12 * diag + extra * diag)
    return err / diag


# ------------------------------------------------------------ decomposition

def test_decompose_single_cubic_exact():
    cs, _ = synth.single_cubic(n_proj=1, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 0.0)
    ref = O.decompose_curves(cs, 0.0)
    seg_off, ctrl, prange = segs.view()
    assert seg_off.tolist() == [0, 13] == ref.seg_off.tolist()
    assert np.array_equal(ctrl, ref.ctrl) and np.array_equal(prange, ref.prange)


@pytest.mark.parametrize("tol", [1e-10, 1e-6])
def test_decompose_curve_set_bit_exact(tol):
    cs, _ = synth.curve_set(seed=2, n_curves=4096, n_proj=1, n_inv=1)
    sub = cs.subset(np.arange(0, 4096, 8))  # 512 curves, all degrees
    segs = bspl.decompose(bspl.DeviceCurves(sub, DEV), tol)
    ref = O.decompose_curves(sub, tol)
    seg_off, ctrl, prange = segs.view()
    assert np.array_equal(seg_off, ref.seg_off)
    assert np.array_equal(prange, ref.prange)
    assert np.array_equal(ctrl, ref.ctrl)


def test_decompose_full_curve_set_counts():
    """The 4,096-curve set at 1e-10 x diag: offsets bit-exact."""
    cs, _ = synth.curve_set(seed=2, n_proj=1, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-10)
    ref = O.decompose_curves(cs, 1e-10, count_only=True)
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)
    # tables: every box holds its cubic's control points
    rec = segs.rec64[: segs.total].cpu().numpy()
    ctrl = segs.ctrl[: segs.total].cpu().numpy()
    assert np.all(rec[:, None, 0:3] <= ctrl) and np.all(ctrl <= rec[:, None, 3:6])


def test_decompose_rejects_invalid():
    U = np.array([0, 0, 0, 0.5, 0.4, 1, 1, 1.0])
    cs = synth.pack_curves([2], [U], [np.zeros((5, 3))])
    with pytest.raises(bspl.BsplError):
        bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-6)


# ------------------------------------------------------------------ queries

@pytest.mark.parametrize("prec", [bspl.FP64, bspl.MIXED])
@pytest.mark.parametrize("samples", [16, 32])
def test_single_cubic_all_queries(prec, samples):
    cs, qs = synth.single_cubic(seed=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 0.0)
    t, d, st = run_queries(segs, qs.proj_curve, qs.proj_xyz, prec=prec, samples=samples)
    check_against_oracle(cs, qs.proj_curve, qs.proj_xyz, t, d, 0.0)
    assert np.all(st & bspl.Q_CONVERGED)
    C, _, _ = O.eval_curves(cs, qs.inv_curve, qs.inv_t)
    t, d, st = run_queries(segs, qs.inv_curve, C, invert=True, prec=prec, samples=samples)
    diag = O.curve_diag(cs)[0]
    assert np.all(d <= 1e-12 * diag)
    assert not np.any(st & bspl.Q_OFF_CURVE)
    check_against_oracle(cs, qs.inv_curve, C, t, d, 0.0)


@pytest.mark.parametrize("prec", [bspl.FP64, bspl.MIXED, bspl.CLIP_MIXED])
def test_curve_set_subset_parity(prec):
    cs, _ = synth.curve_set(seed=2, n_proj=1, n_inv=1)
    sub = cs.subset(np.arange(1, 4096, 16))  # 256 curves
    rng = np.random.default_rng(9)
    lo, hi = synth.cp_boxes(sub)
    qc = rng.integers(0, sub.n, 4000).astype(np.int32)
    q = synth._box_queries(rng, lo, hi, qc)
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(sub, DEV), tol)
    t, d, st = run_queries(segs, qc, q, prec=prec)
    check_against_oracle(sub, qc, q, t, d, tol)
    ic = rng.integers(0, sub.n, 4000).astype(np.int32)
    it = rng.uniform(0, 1, 4000)
    C, _, _ = O.eval_curves(sub, ic, it)
    t, d, st = run_queries(segs, ic, C, invert=True, prec=prec)
    check_against_oracle(sub, ic, C, t, d, tol)
    assert np.all(d <= 1e-9 * O.curve_diag(sub)[ic])


def compare_with_oracle(cs, qc, q, t_o, d_o, t_gpu, d_gpu, tol):
    """check_against_oracle with the oracle's answers computed once."""
    diag = O.curve_diag(cs)[qc]
    err = np.abs(d_gpu - d_o)
    assert np.all(np.isfinite(d_gpu))
    bad = np.where(err > tol * diag + 1e-12 * diag)[0]
    assert len(bad) == 0, (len(bad), err[bad][:5] / diag[bad][:5], qc[bad][:5])
    C, _, _ = O.eval_curves(cs, qc, t_gpu)
    d_orig = np.linalg.norm(C - q, axis=1)
    assert np.all(d_orig <= d_o + 2 * tol * diag + 1e-12 * diag)


def test_full_size_curve_set_oracle_parity():
    """The 4,096-curve set, 1M projection + 1M inversion queries in the launch
    configuration the benchmark times: the plain, mixed, learned and
    clipping-search paths (the learned one captured as a CUDA graph by the
    library and replayed, as the benchmark does) against the oracle on EVERY
    query."""
    cs, qs = synth.curve_set(seed=2)
    tol = 1e-10
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, tol)
    inv_pts = bspl.bspl_eval_curves(dc, dev(qs.inv_curve, torch.int32), dev(qs.inv_t, torch.float64))
    res = {}
    # the learned path with a seed network of random weights (results do not
    # depend on the weights)
    mlp = bspl.Mlp(synth.mlp_init(21))
    pc_d, pq_d, ic_d = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64), dev(qs.inv_curve, torch.int32)
    bp = bspl.QueryBuffers(segs, len(qs.proj_curve), DEV, learned=True)
    bi = bspl.QueryBuffers(segs, len(qs.inv_curve), DEV, learned=True)

    def learned_step():
        o = bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp)
        bspl.bspl_project_curves(segs, pc_d, pq_d, o, bp)
        bspl.bspl_invert_curves(segs, ic_d, inv_pts, o, bi)

    learned_step()
    torch.cuda.synchronize()
    with bspl.Graph() as g:
        learned_step()
    assert g.n_kernels >= 20  # two calls of the learned pipeline
    for x in (bp.dist, bi.dist):
        x.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    assert bspl.mlp_check() == bspl.OK
    res[bspl.LEARNED_MIXED] = tuple(x.cpu().numpy().copy() for x in (bp.param, bp.dist, bp.status, bi.param,
                                                                     bi.dist, bi.status))
    for prec in (bspl.FP64, bspl.MIXED, bspl.CLIP_MIXED):
        tp, dp, sp = run_queries(segs, qs.proj_curve, qs.proj_xyz, prec=prec)
        r = bspl.bspl_invert_curves(segs, dev(qs.inv_curve, torch.int32), inv_pts, bspl.make_options(prec=prec))
        torch.cuda.synchronize()
        res[prec] = (tp, dp, sp, r.param.cpu().numpy().copy(), r.dist.cpu().numpy().copy(),
                     r.status.cpu().numpy().copy())
    diag_i = O.curve_diag(cs)[qs.inv_curve]
    for prec, (tp, dp, sp, ti, di, si) in res.items():
        assert np.all(np.isfinite(dp)) and np.all(np.isfinite(di))
        assert np.all(di <= 1e-9 * diag_i), (prec, np.max(di / diag_i))
        assert not np.any(si & bspl.Q_INVALID) and not np.any(sp & bspl.Q_INVALID)
    # the oracle on every query, once per query set, against all three paths
    inv = inv_pts.cpu().numpy()
    t_op, d_op = O.project_curves(cs, qs.proj_curve, qs.proj_xyz)
    t_oi, d_oi = O.project_curves(cs, qs.inv_curve, inv)
    for prec in (bspl.FP64, bspl.MIXED, bspl.LEARNED_MIXED, bspl.CLIP_MIXED):
        tp, dp, sp, ti, di, si = res[prec]
        compare_with_oracle(cs, qs.proj_curve, qs.proj_xyz, t_op, d_op, tp, dp, tol)
        compare_with_oracle(cs, qs.inv_curve, inv, t_oi, d_oi, ti, di, tol)


def test_learned_16m_projections_vs_plain_and_oracle():
    """The learned-seed workload at its configured size: 16M projection
    queries on the 4,096-curve set.  Learned (trained-or-not does not matter
    for the result) against the plain FP64 path on every query, against the
    oracle on a 100k sample."""
    cs, qs = synth.curve_set(seed=2, n_proj=16_000_000, n_inv=0)
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), tol)
    mlp = bspl.Mlp(synth.mlp_init(21))
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    fast = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp))
    torch.cuda.synchronize()
    t_f, d_f = fast.param.cpu().numpy().copy(), fast.dist.cpu().numpy().copy()
    del fast
    plain = bspl.bspl_project_curves(segs, qc, q, bspl.make_options(prec=bspl.FP64))
    torch.cuda.synchronize()
    d_p = plain.dist.cpu().numpy().copy()
    del plain
    diag = O.curve_diag(cs)[qs.proj_curve]
    rel = np.abs(d_f - d_p) / diag
    assert np.all(np.isfinite(d_f))
    assert rel.max() <= 1e-9, (int((rel > 1e-9).sum()), rel.max(), np.argmax(rel))
    pick = np.random.default_rng(31).choice(len(qc), 100_000, replace=False)
    t_o, d_o = O.project_curves(cs, qs.proj_curve[pick], qs.proj_xyz[pick])
    compare_with_oracle(cs, qs.proj_curve[pick], qs.proj_xyz[pick], t_o, d_o, t_f[pick], d_f[pick], tol)
    assert bspl.mlp_check() == bspl.OK


# --------------------------------------------------------------- edge cases

def _edge_set():
    rng = np.random.default_rng(5)
    curves = []
    curves.append((1, synth.uniform_clamped_knots(1, 2), rng.uniform(0, 1, (2, 3))))  # a single line segment
    curves.append((2, np.array([0, 0, 0, 1, 1, 1.0]), rng.uniform(0, 1, (3, 3))))  # one parabola
    U = np.array([0, 0, 0, 0, 0.3, 0.3, 0.3, 0.7, 1, 1, 1, 1.0])  # C0 join at 0.3
    curves.append((3, U, rng.uniform(0, 1, (8, 3))))
    U = np.array([0, 0, 0, 0, 0, 0, 0.5, 0.5, 0.5, 0.5, 0.5, 1, 1, 1, 1, 1, 1.0])  # degree 5, C0 join
    curves.append((5, U, rng.uniform(0, 1, (11, 3))))
    curves.append((7, synth.uniform_clamped_knots(7, 8), rng.uniform(0, 1, (8, 3))))  # one degree-7 span
    U = np.concatenate([[-3.0] * 4, [-1.0, 2.0], [5.0] * 4])  # non-[0,1] parameter domain
    curves.append((3, U, rng.uniform(0, 1, (6, 3))))
    return synth.pack_curves(*zip(*curves))


@pytest.mark.parametrize("prec", [bspl.FP64, bspl.MIXED, bspl.CLIP_MIXED])
def test_edge_curves(prec):
    cs = _edge_set()
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), tol)
    ref = O.decompose_curves(cs, tol)
    assert np.array_equal(segs.seg_off.cpu().numpy(), ref.seg_off)
    rng = np.random.default_rng(6)
    qc = np.repeat(np.arange(cs.n, dtype=np.int32), 300)
    lo, hi = synth.cp_boxes(cs)
    q = synth._box_queries(rng, lo, hi, qc, scale=2.0)
    # points exactly at control points and curve ends
    ends = []
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        ends += [(c, P[0]), (c, P[-1]), (c, P[len(P) // 2])]
    qc = np.concatenate([qc, np.array([e[0] for e in ends], np.int32)])
    q = np.concatenate([q, np.array([e[1] for e in ends])])
    t, d, st = run_queries(segs, qc, q, prec=prec)
    check_against_oracle(cs, qc, q, t, d, tol)
    p0 = np.array([cs.curve(int(c))[1][cs.curve(int(c))[0]] for c in qc])
    p1 = np.array([cs.curve(int(c))[1][len(cs.curve(int(c))[2])] for c in qc])
    assert np.all((t >= p0) & (t <= p1))


def test_invalid_and_empty_queries():
    cs, qs = synth.single_cubic(n_proj=64, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 0.0)
    qc = qs.proj_curve.copy()
    q = qs.proj_xyz.copy()
    qc[3] = 7  # out of range
    qc[5] = -1
    q[9, 1] = np.nan
    t, d, st = run_queries(segs, qc, q)
    for k in (3, 5, 9):
        assert st[k] == bspl.Q_INVALID and np.isnan(d[k])
    ok = np.setdiff1d(np.arange(64), [3, 5, 9])
    assert np.all(st[ok] & bspl.Q_CONVERGED)
    # empty batch
    r = bspl.bspl_project_curves(segs, dev(np.zeros(0, np.int32), torch.int32),
                                 dev(np.zeros((0, 3)), torch.float64))
    assert r.dist.numel() == 0


def test_counters_and_unsorted_order_agree():
    cs, qs = synth.curve_set(seed=2, n_curves=64, n_proj=3000, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-10)
    cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=DEV)
    t1, d1, _ = run_queries(segs, qs.proj_curve, qs.proj_xyz, counters=cnt)
    t2, d2, _ = run_queries(segs, qs.proj_curve, qs.proj_xyz, sort_queries=0)
    assert np.array_equal(d1, d2) and np.array_equal(t1, t2)
    c = cnt.cpu().numpy()
    assert c[0] == 3000 and c[3] >= 3000 and c[4] >= 3000


def test_near_cusp_segment():
    """A cubic whose last three control points nearly coincide ends in a
    hook where E = (C - q).C' stays below FP32 resolution over a range of u
    and D can have two minima a few hundredths apart in u.  Inversion points
    on the hook must be found at distance ~0 by every path (the FP32 stages
    cannot tell those minima apart; the FP64 stage must)."""
    R = np.array([[0.84270971, 0.61142076, 0.05979669], [0.89519636, 0.69535237, 0.12377618],
                  [0.88879253, 0.68117491, 0.11230443], [0.88830283, 0.68292934, 0.11401205]])
    cs = synth.pack_curves([3], [np.array([0, 0, 0, 0, 1, 1, 1, 1.0])], [R])
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-10)
    t = np.linspace(0.55, 1.0, 20001)
    qc = np.zeros(len(t), np.int32)
    on = O.eval_curves(cs, qc, t)[0]
    rng = np.random.default_rng(31)
    near = on + rng.normal(0, 2e-5, on.shape)
    diag = O.curve_diag(cs)[0]
    mlp = bspl.Mlp(synth.mlp_init(7), DEV)
    _, d_o = O.project_curves(cs, qc, near)
    for prec, kw in ((bspl.FP64, {}), (bspl.LEARNED_MIXED, {"mlp": mlp}), (bspl.LEARNED_MIXED, {}),
                     (bspl.CLIP_MIXED, {})):
        _, d, _ = run_queries(segs, qc, on, invert=True, prec=prec, **kw)
        assert np.max(d) <= 1e-9 * diag, (prec, np.max(d) / diag, t[np.argmax(d)])
        _, d, _ = run_queries(segs, qc, near, prec=prec, **kw)
        assert np.max(np.abs(d - d_o)) <= 1e-9 * diag, (prec, np.max(np.abs(d - d_o)) / diag)
    assert bspl.mlp_check() == bspl.OK
    # the mixed grid path seeds from FP32 samples: two minima closer than
    # the sample spacing form one basin, and its FP64 finish polishes the
    # one FP32 picked (a known limitation of that path; bounded, reported)
    _, d, _ = run_queries(segs, qc, on, invert=True, prec=bspl.MIXED)
    miss = d > 1e-9 * diag
    print(f"mixed grid path, near-cusp inversions: {int(miss.sum())} of {len(t)} off the curve")
    assert miss.mean() < 0.02


def test_learned_single_query_regression():
    """One projection query of the 16M-query workload on the 4,096-curve set
    where the learned path returned the local minimum of another segment
    (0.0778 instead of 0.0719), alone, with and without a network.  On the
    right segment E(1) is 2^-22 in FP32, the size of its rounding: rounded
    to exactly 0, the isolation saw one sign change yet no crossing from -
    to + (it tested the last coefficient, not the last nonzero one) and kept
    the end u = 1, where E' < 0 let the two FP64 steps stop without a step."""
    cs, _ = synth.curve_set(seed=2, n_curves=4096, n_proj=1, n_inv=0)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-10)
    qc = np.array([3673], np.int32)
    q = np.array([[0.23736739375306443, 0.4436718404236332, 0.4354219370688256]])
    _, d_o = O.project_curves(cs, qc, q)
    _, d, _ = run_queries(segs, qc, q, prec=bspl.LEARNED_MIXED)
    assert abs(d[0] - d_o[0]) <= 1e-9 * O.curve_diag(cs)[3673]


def test_graph_captures_in_a_loop():
    """Captures made one after another (each `with Graph() as g` releases
    the previous graph while its own capture is open) replay the same
    results as direct calls, for every curve precision."""
    cs, qs = synth.curve_set(seed=2, n_curves=64, n_proj=5000, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), 1e-10)
    qc, q = dev(qs.proj_curve, torch.int32), dev(qs.proj_xyz, torch.float64)
    mlp = bspl.Mlp(synth.mlp_init(7), DEV)
    g = None
    for prec in (bspl.LEARNED_MIXED, bspl.MIXED, bspl.FP64, bspl.CLIP_MIXED) * 2:
        o = bspl.make_options(prec=prec, mlp=mlp if prec == bspl.LEARNED_MIXED else None)
        bufs = bspl.QueryBuffers(segs, qc.numel(), DEV, learned=prec in (bspl.LEARNED_MIXED, bspl.CLIP_MIXED))
        ref = bspl.bspl_project_curves(segs, qc, q, o).dist.cpu().numpy().copy()
        with bspl.Graph() as g:
            bspl.bspl_project_curves(segs, qc, q, o, bufs)
        bufs.dist.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(bufs.dist.cpu().numpy(), ref), prec
