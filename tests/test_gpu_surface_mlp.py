"""GPU tests of the surface seed network (include/bspl_mlp.h, kind
BSPL_MLP_SURFACE: 48 bicubic coefficients + 3 query coordinates -> (u, v))
through the C ABI: fused tensor-core inference and training gradients
against the FP64 reference (oracle/mlp.py), pair features and labels against
the oracle's, parity of the learned surface path with the oracle and the
plain FP64 path (with a network, and without one), and what training gains."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL_S = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def rand_theta(seed):
    theta = synth.smlp_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    p = M.unpack(theta, M.SHAPES_SURF)
    for b in ("b1", "b2", "b3", "b4"):
        p[b][:] = rng.normal(0, 0.2, p[b].shape)
    return theta


def rand_inputs(rng, n):
    X = np.zeros((n, 64))
    X[:, :48] = rng.uniform(-0.5, 0.5, (n, 48))
    X[:, 48:51] = rng.uniform(-1, 1, (n, 3))
    return X


def test_surface_forward_matches_bf16_reference():
    theta = rand_theta(1)
    m = bspl.Mlp(theta, kind=bspl.MLP_SURFACE)
    rng = np.random.default_rng(2)
    X = rand_inputs(rng, 1000 + 41)  # several tiles and a ragged tail
    t = m.forward(dev(X, torch.float32)).cpu().numpy()
    assert t.shape == (len(X), 2)
    p = M.unpack(theta.astype(np.float32).astype(np.float64), M.SHAPES_SURF)
    ref16 = M.forward(p, X.astype(np.float32), bf16=True)[0]
    # the reference rounds weights and layer inputs to BF16; the kernel also
    # evaluates GELU in packed BF16 arithmetic (five roundings per value)
    assert np.max(np.abs(t - ref16)) < 4e-3, np.max(np.abs(t - ref16))
    assert np.max(np.abs(t - M.forward(p, X)[0])) < 1e-2
    assert bspl.mlp_check() == bspl.OK


def test_surface_loss_and_gradients_match_reference():
    theta = rand_theta(3)
    m = bspl.Mlp(theta, kind=bspl.MLP_SURFACE)
    rng = np.random.default_rng(4)
    n = 2500
    X = rand_inputs(rng, n)
    y = rng.uniform(0, 1, (n, 2))
    loss, grad = m.loss_grad(dev(X, torch.float32), dev(y, torch.float32))
    loss, grad = float(loss.item()), grad.cpu().numpy().astype(np.float64)
    p = M.unpack(theta.astype(np.float32).astype(np.float64), M.SHAPES_SURF)
    ref_loss, g = M.loss_and_grads(p, X, y)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    G = M.unpack(grad, M.SHAPES_SURF)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        err = np.linalg.norm(G[name] - g[name]) / np.linalg.norm(g[name])
        assert err < 3e-2, (name, err)
    assert np.all(G["W1"][:, 51:] == 0)
    assert np.all(grad[-2:] == 0)
    assert bspl.mlp_check() == bspl.OK


def test_surface_checkpoint_round_trip(tmp_path):
    m = bspl.Mlp(rand_theta(7), kind=bspl.MLP_SURFACE)
    m.adam(torch.full((bspl.SMLP_NPARAM,), 1e-3, device=DEV), lr=1e-3)
    path = tmp_path / "sseed.bin"
    m.save(path)
    m2 = bspl.Mlp.load(path)
    assert m2.kind == bspl.MLP_SURFACE and m2.step == 1
    assert torch.equal(m.params, m2.params) and torch.equal(m.wbf16, m2.wbf16)


def _surface_batch(n_surf=24, n_q=3000, seed=11):
    ss, _ = synth.surface_set(seed=3, n_surf=n_surf, n_proj=1, n_inv=1, n_range=(6, 12))
    rng = np.random.default_rng(seed)
    qs = rng.integers(0, ss.n, n_q).astype(np.int32)
    S = O.eval_surfaces(ss, qs, rng.uniform(0, 1, (n_q, 2)))[0]
    w = synth.sphere_dirs(rng, n_q)
    r = rng.uniform(0, 0.2, n_q) * O.surface_diag(ss)[qs]
    return ss, qs, S + w * r[:, None], S


def test_surface_pairs_features_and_labels():
    ss, qs, q, _ = _surface_batch()
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), TOL_S)
    qd = dev(q, torch.float64)
    pq, pp, found = bspl.bspl_smlp_collect_pairs(segs, dev(qs, torch.int32), qd, cap=200_000)
    assert 0 < pq.numel() <= found
    pq_h, pp_h = pq.cpu().numpy(), pp.cpu().numpy()
    # every pair's patch belongs to its query's surface
    seg_off = segs.seg_off.cpu().numpy()
    assert np.all((pp_h >= seg_off[qs[pq_h]]) & (pp_h < seg_off[qs[pq_h] + 1]))
    X = bspl.bspl_smlp_features(segs, pq, pp, qd).cpu().numpy()
    uv = bspl.bspl_smlp_labels(segs, pq, pp, qd).cpu().numpy()
    ctrl = segs.ctrl[: segs.total].cpu().numpy()
    k = np.random.default_rng(1).choice(len(pq_h), min(300, len(pq_h)), replace=False)
    Xo = M.surface_features(ctrl[pp_h[k]], q[pq_h[k]])
    assert np.max(np.abs(X[k] - Xo)) < 2e-4, np.max(np.abs(X[k] - Xo))
    # labels: the minimiser of the pair's bicubic (distances compared: ties)
    for j in k[:120]:
        P = ctrl[pp_h[j]]
        u, v, D = M.patch_minimiser(P, q[pq_h[j]], samples=17)
        Dg = float(np.sum((M._patch(P, uv[j, 0], uv[j, 1]) - q[pq_h[j]]) ** 2))
        assert Dg <= D + 1e-6 * (1 + D), (j, Dg, D)


@pytest.mark.parametrize("net", ["none", "untrained"])
def test_learned_surface_parity(net):
    """The learned surface path with no network (seed = patch centre) and
    with random weights: the same answers as the plain FP64 path on every
    query and the oracle on a sample (the certification does not depend on
    the seed)."""
    ss, qs, q, on = _surface_batch(n_surf=32, n_q=6000, seed=12)
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), TOL_S)
    mlp = None if net == "none" else bspl.Mlp(rand_theta(13), kind=bspl.MLP_SURFACE)
    diag = O.surface_diag(ss)[qs]
    for pts, fn in ((q, bspl.bspl_project_surfaces), (on, bspl.bspl_invert_surfaces)):
        qd, sd = dev(pts, torch.float64), dev(qs, torch.int32)
        cnt = torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=DEV)
        r = fn(segs, sd, qd, bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp, counters=cnt))
        torch.cuda.synchronize()
        d_l, uv_l = r.dist.cpu().numpy().copy(), r.param.cpu().numpy().copy()
        d_p = fn(segs, sd, qd, bspl.make_options(prec=bspl.FP64)).dist.cpu().numpy()
        assert np.all(np.isfinite(d_l))
        rel = np.abs(d_l - d_p) / diag
        assert rel.max() <= 1e-9, (int((rel > 1e-9).sum()), rel.max())
        c = dict(zip(bspl.COUNTER_NAMES, cnt.cpu().tolist()))
        assert c["queries"] == len(qs) and c["candidates"] > 0
        pick = np.random.default_rng(2).choice(len(qs), 600, replace=False)
        _, d_o = O.project_surfaces(ss, qs[pick], pts[pick])
        assert np.max(np.abs(d_l[pick] - d_o) / diag[pick]) <= 1e-9
        S = O.eval_surfaces(ss, qs[pick], uv_l[pick])[0]
        assert np.all(np.abs(np.linalg.norm(S - pts[pick], axis=1) - d_l[pick]) <= 1e-9 * diag[pick])
    assert bspl.mlp_check() == bspl.OK


def test_surface_training_gain():
    """Trained on (query, patch) pairs of one surface set, labelled by the
    pair's minimiser: on the pairs of another the network's seed is closer
    to the minimiser than the patch centre."""
    ss, qs, q, _ = _surface_batch(n_surf=48, n_q=40000, seed=21)
    segs = bspl.decompose(bspl.DeviceSurfaces(ss, DEV), TOL_S)
    qd = dev(q, torch.float64)
    pq, pp, _ = bspl.bspl_smlp_collect_pairs(segs, dev(qs, torch.int32), qd, cap=2_000_000)
    X = bspl.bspl_smlp_features(segs, pq, pp, qd)
    y = bspl.bspl_smlp_labels(segs, pq, pp, qd)
    n = X.shape[0]
    tr, te = slice(0, int(0.8 * n)), slice(int(0.8 * n), n)
    m = bspl.Mlp(synth.smlp_init(8), kind=bspl.MLP_SURFACE)
    loss = m.train(X[tr].contiguous(), y[tr].contiguous(), epochs=4, batch=4096, lr=2e-3, seed=3).cpu().numpy()
    err_net = (m.forward(X[te].contiguous()) - y[te]).abs().mean().item()
    err_mid = (0.5 - y[te]).abs().mean().item()
    print(f"surface seed |uv - uv*|: network {err_net:.4f}, patch centre {err_mid:.4f}; "
          f"training loss {loss[0]:.5f} -> {loss[-1]:.5f}")
    assert loss[-1] < loss[0]
    assert err_net < 0.8 * err_mid
    assert bspl.mlp_check() == bspl.OK
