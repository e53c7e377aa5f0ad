"""GPU tests of the learned Newton seed (include/bspl_mlp.h) through the C ABI:
the fused tensor-core inference and the training kernels against the FP64
reference (oracle/mlp.py), the pair collection, features and labels against
the oracle's decomposition, parity of the learned path with the projection
oracle with and without a network, and what the trained network gains."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth
from test_gpu_curves import check_against_oracle

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def rand_theta(seed):
    theta = synth.mlp_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    p = M.unpack(theta)
    for b in ("b1", "b2", "b3", "b4"):
        p[b][:] = rng.normal(0, 0.2, p[b].shape)
    return theta


def rand_inputs(rng, n):
    X = np.zeros((n, 16))
    X[:, :12] = rng.uniform(-0.5, 0.5, (n, 12))
    v = rng.normal(size=(n, 3))
    X[:, 12:15] = v / np.maximum(1, np.linalg.norm(v, axis=1))[:, None]
    return X


def test_fused_forward_matches_bf16_reference():
    theta = rand_theta(1)
    m = bspl.Mlp(theta)
    rng = np.random.default_rng(2)
    X = rand_inputs(rng, 1000 + 37)  # several tiles and a ragged tail
    t = m.forward(dev(X, torch.float32)).cpu().numpy()
    p = M.unpack(theta.astype(np.float32).astype(np.float64))
    ref16 = M.forward(p, X.astype(np.float32), bf16=True)[0]
    ref = M.forward(p, X)[0]
    # the reference rounds weights and layer inputs to BF16; the kernel also
    # evaluates GELU in packed BF16 arithmetic (five roundings per value)
    assert np.max(np.abs(t - ref16)) < 4e-3, np.max(np.abs(t - ref16))
    assert np.max(np.abs(t - ref)) < 1e-2
    assert bspl.mlp_check() == bspl.OK


def test_training_loss_and_gradients_match_reference():
    theta = rand_theta(3)
    m = bspl.Mlp(theta)
    rng = np.random.default_rng(4)
    n = 3000  # not a multiple of the 128-row tile
    X = rand_inputs(rng, n)
    y = rng.uniform(0, 1, n)
    loss, grad = m.loss_grad(dev(X, torch.float32), dev(y, torch.float32))
    loss, grad = float(loss.item()), grad.cpu().numpy().astype(np.float64)
    p = M.unpack(theta.astype(np.float32).astype(np.float64))
    ref_loss, g = M.loss_and_grads(p, X, y)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    G = M.unpack(grad)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        err = np.linalg.norm(G[name] - g[name]) / np.linalg.norm(g[name])
        assert err < 3e-2, (name, err)
    assert np.all(G["W1"][:, 15] == 0)
    assert np.all(grad[-3:] == 0)
    assert bspl.mlp_check() == bspl.OK


def test_adam_matches_reference_and_refreshes_bf16_copy():
    theta = rand_theta(5)
    m = bspl.Mlp(theta)
    rng = np.random.default_rng(6)
    th, mm, vv = theta.astype(np.float32).astype(np.float64), np.zeros(M.NPARAM), np.zeros(M.NPARAM)
    for k in (1, 2, 3):
        g = rng.normal(0, 1e-2, M.NPARAM).astype(np.float32)
        m.adam(dev(g, torch.float32), lr=1e-3)
        th, mm, vv = M.adam(th, g.astype(np.float64), mm, vv, k, 1e-3)
    got = m.params.cpu().numpy()
    assert np.max(np.abs(got - th)) < 1e-6
    # the BF16 copy follows the master weights
    X = rand_inputs(rng, 256)
    t = m.forward(dev(X, torch.float32)).cpu().numpy()
    ref16 = M.forward(M.unpack(got.astype(np.float64)), X.astype(np.float32), bf16=True)[0]
    assert np.max(np.abs(t - ref16)) < 4e-3  # packed BF16 GELU, as in the forward test


def test_checkpoint_round_trip(tmp_path):
    m = bspl.Mlp(rand_theta(7))
    m.adam(torch.full((bspl.MLP_NPARAM,), 1e-3, device=DEV), lr=1e-3)
    path = tmp_path / "seed.bin"
    m.save(path)
    m2 = bspl.Mlp.load(path)
    assert m2.step == 1
    for a, b in ((m.params, m2.params), (m.adam_m, m2.adam_m), (m.adam_v, m2.adam_v), (m.wbf16, m2.wbf16)):
        assert torch.equal(a, b)
    raw = bytearray(path.read_bytes())
    raw[-1] ^= 1
    path.write_bytes(bytes(raw))
    with pytest.raises(bspl.BsplError):
        bspl.Mlp.load(path)


def _subset(n_curves=256, n_q=4000, seed=9, stride_seed=2):
    cs, _ = synth.curve_set(seed=stride_seed, n_proj=1, n_inv=1)
    sub = cs.subset(np.arange(1, 4096, 4096 // n_curves))
    rng = np.random.default_rng(seed)
    lo, hi = synth.cp_boxes(sub)
    qc = rng.integers(0, sub.n, n_q).astype(np.int32)
    q = synth._box_queries(rng, lo, hi, qc)
    ic = rng.integers(0, sub.n, n_q).astype(np.int32)
    C, _, _ = O.eval_curves(sub, ic, rng.uniform(0, 1, n_q))
    return sub, qc, q, ic, C


def test_collect_pairs_features_and_labels():
    sub, qc, q, _, _ = _subset(n_q=20000)
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(sub, DEV), tol)
    qd = dev(q, torch.float64)
    pq, ps, n = bspl.bspl_mlp_collect_pairs(segs, dev(qc, torch.int32), qd, cap=400_000)
    assert 0 < n <= 400_000 and pq.numel() == n
    # a small capacity writes a prefix and still reports the pairs found (the
    # count can differ by a few: a candidate is filtered against its query's
    # bound as it stands when the warp's shared buffer is classified, and the
    # queries sharing a warp vary with the order inside a curve's bucket)
    pq2, ps2, n2 = bspl.bspl_mlp_collect_pairs(segs, dev(qc, torch.int32), qd, cap=n // 3)
    assert abs(n2 - n) <= n // 100 and 0 < pq2.numel() <= n // 3
    ref = O.decompose_curves(sub, tol)
    pqn, psn = pq.cpu().numpy(), ps.cpu().numpy()
    assert np.all(qc[pqn] >= 0)
    # every seeded segment belongs to its query's curve
    assert np.all((psn >= ref.seg_off[qc[pqn]]) & (psn < ref.seg_off[qc[pqn] + 1]))
    P = ref.ctrl[psn]
    qq = q[pqn]
    # the certified class: E(0) < 0 < E(1), one minimum inside the segment
    E0 = np.einsum("ij,ij->i", P[:, 0] - qq, P[:, 1] - P[:, 0])
    E1 = np.einsum("ij,ij->i", P[:, 3] - qq, P[:, 3] - P[:, 2])
    assert np.all(E0 < 0) and np.all(E1 > 0)
    X = bspl.bspl_mlp_features(segs, pq, ps, qd).cpu().numpy()
    # FP32 inputs: a few ulps of the query's distance in segment units
    lo, hi = P.min(1), P.max(1)
    vn = np.linalg.norm(qq - 0.5 * (lo + hi), axis=1) / (hi - lo).max(1)
    err = np.abs(X - M.features(P, qq)).max(1)
    assert np.all(err <= 1e-4 + 2e-6 * vn), np.max(err / (1e-4 + 2e-6 * vn))
    y = bspl.bspl_mlp_labels(segs, pq, ps, qd).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    pick = rng.choice(n, min(n, 400), replace=False)
    far = 0
    for i in pick:
        u, D = M.segment_minimiser(P[i], qq[i])
        Dg = float(np.sum((M._bezier(P[i], np.array([y[i]]))[0] - qq[i]) ** 2))
        assert Dg <= D + 1e-12 * (1 + D)
        far += abs(y[i] - u) > 1e-4
    assert far <= 2


def _counters():
    return torch.zeros(bspl.NCOUNTERS, dtype=torch.int64, device=DEV)


def _run(segs, qc, q, invert, prec, mlp=None, ctr=None):
    fn = bspl.bspl_invert_curves if invert else bspl.bspl_project_curves
    r = fn(segs, dev(qc, torch.int32), dev(q, torch.float64), bspl.make_options(prec=prec, mlp=mlp, counters=ctr))
    torch.cuda.synchronize()
    return r.param.cpu().numpy().copy(), r.dist.cpu().numpy().copy(), r.status.cpu().numpy().copy()


@pytest.mark.parametrize("net", ["none", "untrained"])
def test_learned_path_parity(net):
    """Correctness does not rest on the network: without one (seed 1/2) and
    with random weights the learned path matches the oracle on every query."""
    sub, qc, q, ic, C = _subset()
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(sub, DEV), tol)
    mlp = None if net == "none" else bspl.Mlp(rand_theta(11))
    ctr = _counters()
    t, d, st = _run(segs, qc, q, False, bspl.LEARNED_MIXED, mlp, ctr)
    check_against_oracle(sub, qc, q, t, d, tol)
    # the two FP64 steps settle almost every query; the FP64 fallback (the
    # certified FP64 isolation, also taken by pairs whose FP32 isolation was
    # uncertain or could not separate two candidates) decides a few percent
    assert int(ctr[bspl.COUNTER_NAMES.index("fallback")]) <= 3 * len(qc) // 100
    assert not np.any(st & (bspl.Q_INVALID | bspl.Q_NONCONV))
    t, d, st = _run(segs, ic, C, True, bspl.LEARNED_MIXED, mlp)
    check_against_oracle(sub, ic, C, t, d, tol)
    assert np.all(d <= 1e-9 * O.curve_diag(sub)[ic])
    assert not np.any(st & (bspl.Q_INVALID | bspl.Q_NONCONV))
    # and agrees with the grid path on every query
    _, dm, _ = _run(segs, qc, q, False, bspl.MIXED)
    _, dl, _ = _run(segs, qc, q, False, bspl.LEARNED_MIXED, mlp)
    assert np.all(np.abs(dm - dl) <= 1e-9 * O.curve_diag(sub)[qc])
    assert bspl.mlp_check() == bspl.OK


def train_seed_network(n_curves=512, n_q=1_000_000, epochs=8, seed=12):
    """Pairs from a curve set disjoint from the test curves (another seed of
    the same recipe), labelled by the FP64 plain solver, then training."""
    cs, qs = synth.curve_set(seed=seed, n_curves=n_curves, n_proj=n_q // 2, n_inv=n_q // 2)
    dc = bspl.DeviceCurves(cs, DEV)
    segs = bspl.decompose(dc, 1e-10)
    inv = bspl.bspl_eval_curves(dc, dev(qs.inv_curve, torch.int32), dev(qs.inv_t, torch.float64))
    qc = torch.cat([dev(qs.proj_curve, torch.int32), dev(qs.inv_curve, torch.int32)])
    q = torch.cat([dev(qs.proj_xyz, torch.float64), inv])
    pq, ps, n = bspl.bspl_mlp_collect_pairs(segs, qc, q, cap=4 * n_q)
    X = bspl.bspl_mlp_features(segs, pq, ps, q)
    y = bspl.bspl_mlp_labels(segs, pq, ps, q)
    m = bspl.Mlp(synth.mlp_init(7))
    loss = m.train(X, y, epochs=epochs, batch=4096, lr=2e-3, seed=5).cpu().numpy()
    return m, loss, n


def test_training_gain_over_the_method_without_it():
    m, loss, npairs = train_seed_network()
    assert npairs > 50_000
    assert loss[-1] < 0.5 * loss[0], loss
    sub, qc, q, ic, C = _subset()
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(sub, DEV), tol)
    # held-out seed error on the test curves' pairs
    qd = dev(q, torch.float64)
    pq, ps, n = bspl.bspl_mlp_collect_pairs(segs, dev(qc, torch.int32), qd, cap=400_000)
    ystar = bspl.bspl_mlp_labels(segs, pq, ps, qd)
    pred = m.forward(bspl.bspl_mlp_features(segs, pq, ps, qd))
    err_net = float(torch.mean(torch.abs(pred - ystar)).item())
    err_mid = float(torch.mean(torch.abs(0.5 - ystar)).item())
    # Newton work with and without the network, results checked both ways
    stats = {}
    for name, mlp in (("none", None), ("trained", m)):
        ctr = _counters()
        t, d, st = _run(segs, qc, q, False, bspl.LEARNED_MIXED, mlp, ctr)
        check_against_oracle(sub, qc, q, t, d, tol)
        t, d, st = _run(segs, ic, C, True, bspl.LEARNED_MIXED, mlp, ctr)
        check_against_oracle(sub, ic, C, t, d, tol)
        stats[name] = dict(zip(bspl.COUNTER_NAMES, ctr.cpu().numpy().tolist()))
    print(f"\nseed error |t - t*|: network {err_net:.4f}, midpoint {err_mid:.4f}; "
          f"FP32 Newton iterations: network {stats['trained']['newton32_iters']}, "
          f"midpoint {stats['none']['newton32_iters']}; training loss {loss[0]:.4g} -> {loss[-1]:.4g}")
    assert err_net < 0.5 * err_mid
    assert stats["trained"]["newton32_iters"] < stats["none"]["newton32_iters"]
    assert bspl.mlp_check() == bspl.OK


def test_learned_path_edge_cases_invalid_and_leftovers():
    """Degenerate and ragged curves, points on control points and ends,
    invalid queries, an empty batch, and a pair buffer too small for most
    queries (they are answered by the grid kernel): oracle parity."""
    from test_gpu_curves import _edge_set
    cs = _edge_set()
    tol = 1e-10
    segs = bspl.decompose(bspl.DeviceCurves(cs, DEV), tol)
    rng = np.random.default_rng(16)
    qc = np.repeat(np.arange(cs.n, dtype=np.int32), 200)
    lo, hi = synth.cp_boxes(cs)
    q = synth._box_queries(rng, lo, hi, qc, scale=2.0)
    ends = []
    for c in range(cs.n):
        _, _, P = cs.curve(c)
        ends += [(c, P[0]), (c, P[-1]), (c, P[len(P) // 2])]
    qc = np.concatenate([qc, np.array([e[0] for e in ends], np.int32)])
    q = np.concatenate([q, np.array([e[1] for e in ends])])
    mlp = bspl.Mlp(rand_theta(13))
    for ppq in (0, 1):
        ctr = _counters()
        r = bspl.bspl_project_curves(segs, dev(qc, torch.int32), dev(q, torch.float64),
                                     bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp, counters=ctr,
                                                       pairs_per_query=ppq))
        torch.cuda.synchronize()
        check_against_oracle(cs, qc, q, r.param.cpu().numpy(), r.dist.cpu().numpy(), tol)
        if ppq == 1:  # most queries found more than one candidate pair
            assert int(ctr[bspl.COUNTER_NAMES.index("candidates")]) < 2 * len(qc)
    bad_c, bad_q = qc[:6].copy(), q[:6].copy()
    bad_c[1], bad_c[2] = cs.n, -3
    bad_q[4, 2] = np.inf
    r = bspl.bspl_project_curves(segs, dev(bad_c, torch.int32), dev(bad_q, torch.float64),
                                 bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp))
    st = r.status.cpu().numpy()
    assert st[1] == st[2] == st[4] == bspl.Q_INVALID
    assert np.all(st[[0, 3, 5]] & bspl.Q_CONVERGED)
    r = bspl.bspl_project_curves(segs, dev(np.zeros(0, np.int32), torch.int32), dev(np.zeros((0, 3)), torch.float64),
                                 bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp))
    assert r.dist.numel() == 0
