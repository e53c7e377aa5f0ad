"""GPU parity of surface decomposition and surface projection/inversion,
through the C ABI, against the CPU oracle.

Decomposition: patch counts, offsets, bicubic nets and parameter boxes
bit-exact.  Queries: the last Newton steps run on the original span-pair
patch and the certification search bounds D on the original surface, so
|d_gpu - d_oracle| <= 1e-9 x diag for every query whatever the
decomposition tolerance, and the GPU (u, v), evaluated on the original
surface by the oracle, reproduces the GPU distance.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL_S = 1e-4  # surface decomposition tolerance (the paper's alpha, Sec. 5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def small_surface_set(seed=3, n=24):
    ss, _ = synth.surface_set(seed=seed, n_surf=n, n_proj=1, n_inv=1, n_range=(6, 12))
    return ss


def run(segs, qs, q, invert=False, **kw):
    fn = bspl.bspl_invert_surfaces if invert else bspl.bspl_project_surfaces
    r = fn(segs, dev(qs, torch.int32), dev(q, torch.float64), bspl.make_options(**kw))
    torch.cuda.synchronize()
    return r.param.cpu().numpy().copy(), r.dist.cpu().numpy().copy(), r.status.cpu().numpy().copy()


def check(ss, qs, q, uv, d, bound=1e-9):
    uv_o, d_o = O.project_surfaces(ss, qs, q)
    diag = O.surface_diag(ss)[qs]
    assert np.all(np.isfinite(d))
    err = np.abs(d - d_o) / diag
    bad = np.where(err > bound)[0]
    assert len(bad) == 0, (len(bad), err[bad][:5], qs[bad][:5])
    S = O.eval_surfaces(ss, qs, uv)[0]
    assert np.all(np.abs(np.linalg.norm(S - q, axis=1) - d) <= 1e-9 * diag)


def surface_queries(ss, rng, n):
    qs = rng.integers(0, ss.n, n).astype(np.int32)
    uv = rng.uniform(0, 1, (n, 2))
    S = O.eval_surfaces(ss, qs, uv)[0]
    w = synth.sphere_dirs(rng, n)
    r = rng.uniform(0, 0.2, n) * O.surface_diag(ss)[qs]
    return qs, S + w * r[:, None], S


@pytest.mark.parametrize("tol", [TOL_S, 1e-6])
def test_surface_decomposition_bit_exact(tol):
    ss = small_surface_set()
    if tol < 1e-5:  # the tight tolerance only on surfaces with at most one reduced direction
        keep = [s for s in range(ss.n) if not (ss.deg_u[s] > 3 and ss.deg_v[s] > 3)]
        ss = ss.subset(keep)
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), tol)
    ref = O.decompose_surfaces(ss, tol)
    seg_off, ctrl, prange = segs.view()
    assert np.array_equal(seg_off, ref.seg_off)
    assert np.array_equal(prange, ref.prange)
    assert np.array_equal(ctrl, ref.ctrl)


@pytest.mark.parametrize("prec", [bspl.FP64, bspl.MIXED])
def test_surface_projection_and_inversion_parity(prec):
    ss = small_surface_set()
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), TOL_S)
    rng = np.random.default_rng(11)
    qs, q, on = surface_queries(ss, rng, 600)
    uv, d, st = run(segs, qs, q, prec=prec)
    check(ss, qs, q, uv, d)
    assert np.all(st & bspl.Q_CONVERGED)
    uv, d, st = run(segs, qs, on, invert=True, prec=prec)
    diag = O.surface_diag(ss)[qs]
    assert np.all(d <= 1e-9 * diag), np.max(d / diag)
    assert not np.any(st & bspl.Q_OFF_CURVE)


def test_surface_planar_rectangle_closed_form():
    """Greville nets reproduce the rectangle o + R (u Lx, v Ly, 0) (bilinear
    precision), so the projection has a closed form, boundary cases included."""
    rng = np.random.default_rng(25)
    pu, pv, nu, nv = 3, 2, 7, 6
    U = synth.random_clamped_knots(rng, pu, nu, 0.0)
    V = synth.random_clamped_knots(rng, pv, nv, 0.0)
    Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    o, Lx, Ly = rng.uniform(-1, 1, 3), 1.3, 0.7
    gu = np.array([np.mean(U[i + 1:i + pu + 1]) for i in range(nu)])
    gv = np.array([np.mean(V[i + 1:i + pv + 1]) for i in range(nv)])
    P = np.array([[o + Rm @ np.array([a * Lx, b * Ly, 0.0]) for b in gv] for a in gu])
    ss = synth.pack_surfaces([pu], [pv], [U], [V], [P])
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), 1e-10)
    q = o + rng.uniform(-1, 2, (500, 3))
    for prec in (bspl.FP64, bspl.MIXED):
        uv, d, _ = run(segs, np.zeros(500, np.int32), q, prec=prec)
        loc = (q - o) @ Rm
        us, vs = np.clip(loc[:, 0] / Lx, 0, 1), np.clip(loc[:, 1] / Ly, 0, 1)
        ref = np.linalg.norm(loc - np.stack([us * Lx, vs * Ly, 0 * us], 1), axis=1)
        assert np.abs(d - ref).max() <= 1e-12 * 4


def test_surface_edge_cases_and_invalid():
    rng = np.random.default_rng(13)
    nets, KU, KV, pus, pvs = [], [], [], [], []
    # bilinear single patch, a C0 crease in u, and a (5,4) surface
    for pu, pv, nu, nv, U in ((1, 1, 2, 2, None), (3, 2, 7, 5, np.array([0, 0, 0, 0, .5, .5, .5, 1, 1, 1, 1.0])),
                              (5, 4, 8, 7, None)):
        if U is None:
            U = synth.random_clamped_knots(rng, pu, nu, 0.0)
        KU.append(U)
        KV.append(synth.random_clamped_knots(rng, pv, nv, 0.0))
        nets.append(synth._sinusoid_net(rng, nu, nv))
        pus.append(pu)
        pvs.append(pv)
    ss = synth.pack_surfaces(pus, pvs, KU, KV, nets)
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), TOL_S)
    qs, q, on = surface_queries(ss, rng, 300)
    # plus control points and corners
    extra = [(s, ss.surface(s)[4][i, j]) for s in range(ss.n) for i, j in ((0, 0), (-1, -1), (1, 1))]
    qs = np.concatenate([qs, np.array([e[0] for e in extra], np.int32)])
    q = np.concatenate([q, np.array([e[1] for e in extra])])
    for prec in (bspl.FP64, bspl.MIXED):
        uv, d, st = run(segs, qs, q, prec=prec)
        check(ss, qs, q, uv, d)
    bad_q = q[:4].copy()
    bad_s = np.array([0, 9, -2, 1], np.int32)
    bad_q[3, 0] = np.inf
    uv, d, st = run(segs, bad_s, bad_q)
    assert st[1] == bspl.Q_INVALID and st[2] == bspl.Q_INVALID and st[3] == bspl.Q_INVALID
    assert st[0] & bspl.Q_CONVERGED


def test_surface_set_sampled():
    """128 surfaces of the random-surface workload at the paper's alpha:
    200k projection + 200k inversion queries through the kernels, oracle
    parity on a sample of 1,000 per precision, inversion bound and
    mixed-vs-plain agreement on every query."""
    ss, sq = synth.surface_set(seed=3, n_surf=128, n_proj=200_000, n_inv=200_000)
    dsf = bspl.DeviceSurfaces(ss, DEV)
    segs = bspl.decompose(dsf, TOL_S)
    ps = dev(sq.proj_surf, torch.int32)
    base = bspl.bspl_eval_surfaces(dsf, ps, dev(sq.proj_uv, torch.float64))
    q = base + dev(sq.proj_dir, torch.float64) * dev(sq.proj_r, torch.float64)[:, None]
    isf = dev(sq.inv_surf, torch.int32)
    on = bspl.bspl_eval_surfaces(dsf, isf, dev(sq.inv_uv, torch.float64))
    res = {}
    for prec in (bspl.FP64, bspl.MIXED):
        rp = bspl.bspl_project_surfaces(segs, ps, q, bspl.make_options(prec=prec))
        ri = bspl.bspl_invert_surfaces(segs, isf, on, bspl.make_options(prec=prec))
        torch.cuda.synchronize()
        res[prec] = [x.cpu().numpy().copy() for x in (rp.param, rp.dist, ri.param, ri.dist)]
    diag_p = O.surface_diag(ss)[sq.proj_surf]
    diag_i = O.surface_diag(ss)[sq.inv_surf]
    for prec in res:
        assert np.all(res[prec][3] <= 1e-9 * diag_i), np.max(res[prec][3] / diag_i)
    # mixed vs plain on every query (both certified on the original surface)
    rel = np.abs(res[bspl.FP64][1] - res[bspl.MIXED][1]) / diag_p
    assert np.all(rel <= 1e-9), (int((rel > 1e-9).sum()), rel.max())
    rel = np.abs(res[bspl.FP64][3] - res[bspl.MIXED][3]) / diag_i
    assert np.all(rel <= 1e-9), (int((rel > 1e-9).sum()), rel.max())
    rng = np.random.default_rng(4)
    pick = rng.choice(len(sq.proj_surf), 1000, replace=False)
    qn = q.cpu().numpy()
    for prec in res:
        check(ss, sq.proj_surf[pick], qn[pick], res[prec][0][pick], res[prec][1][pick])


def test_certification_counters_and_switch():
    """The certification search runs by default (its cells and leaves are
    counted), can be switched off for timing comparisons (cert_depth < 0),
    and rejects depths above 4."""
    ss, sq = synth.surface_set(seed=3, n_surf=16, n_proj=20_000, n_inv=1)
    dsf = bspl.DeviceSurfaces(ss, DEV)
    segs = bspl.decompose(dsf, TOL_S)
    ps = dev(sq.proj_surf, torch.int32)
    q = bspl.bspl_eval_surfaces(dsf, ps, dev(sq.proj_uv, torch.float64)) + \
        dev(sq.proj_dir, torch.float64) * dev(sq.proj_r, torch.float64)[:, None]
    names = bspl.COUNTER_NAMES
    for prec in (bspl.FP64, bspl.MIXED):
        got = {}
        for cd in (-1, 0, 3):
            cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=DEV)
            bspl.bspl_project_surfaces(segs, ps, q, bspl.make_options(prec=prec, cert_depth=cd, counters=cnt))
            got[cd] = dict(zip(names, cnt.cpu().tolist()))
        assert got[-1]["cert_cells"] == 0 and got[-1]["cert_leaves"] == 0
        assert got[0]["cert_cells"] > 0
        assert got[3]["cert_cells"] >= got[0]["cert_cells"]
        assert got[0]["queries"] == len(sq.proj_surf)
    with pytest.raises(bspl.BsplError, match="EINVAL"):
        bspl.bspl_project_surfaces(segs, ps, q, bspl.make_options(cert_depth=5))
