"""The 1,024-surface set at full size (4M projection + 4M inversion queries,
decomposed at the paper's alpha = 1e-4) through the plain FP64 path and the
fast paths (mixed grid seed, learned seed with an untrained network: the
certification does not depend on the seed).

Every query: fast vs plain within 1e-9 x diag, inversion distances ~0.  The
plain path against the oracle on a stratified subset: every projection
query where a fast path differs from it by more than 1e-11 x diag, every
query a fast path answered through its FP64 fallback (80,000 of those at
most, drawn at random when there are more), and 20,000 random others.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2504_11498_gb300 import bspl, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
ALPHA = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_11498_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=DEV)


def test_full_surface_set_fast_vs_plain_and_oracle():
    ss, sq = synth.surface_set(seed=3)
    dsf = bspl.DeviceSurfaces(ss, DEV)
    segs = bspl.decompose(dsf, ALPHA)
    ps, isf = dev(sq.proj_surf, torch.int32), dev(sq.inv_surf, torch.int32)
    q = bspl.bspl_eval_surfaces(dsf, ps, dev(sq.proj_uv, torch.float64)) + \
        dev(sq.proj_dir, torch.float64) * dev(sq.proj_r, torch.float64)[:, None]
    on = bspl.bspl_eval_surfaces(dsf, isf, dev(sq.inv_uv, torch.float64))
    diag = O.surface_diag(ss)
    smlp = bspl.Mlp(synth.smlp_init(8), DEV, kind=bspl.MLP_SURFACE)
    runs = {}
    for name, prec, net in (("plain", bspl.FP64, None), ("mixed", bspl.MIXED, None),
                            ("learned", bspl.LEARNED_MIXED, smlp)):
        o = bspl.make_options(prec=prec, mlp=net)
        rp = bspl.bspl_project_surfaces(segs, ps, q, o)
        ri = bspl.bspl_invert_surfaces(segs, isf, on, o)
        torch.cuda.synchronize()
        runs[name] = [x.cpu().numpy().copy() for x in (rp.param, rp.dist, rp.status, ri.dist)]
    dp, di = diag[sq.proj_surf], diag[sq.inv_surf]
    for name in runs:
        assert np.all(np.isfinite(runs[name][1]))
        assert np.all(runs[name][3] <= 1e-9 * di), (name, np.max(runs[name][3] / di))
    suspect = np.zeros(len(dp), bool)
    for name in ("mixed", "learned"):
        rel = np.abs(runs[name][1] - runs["plain"][1]) / dp
        assert np.all(rel <= 1e-9), (name, int((rel > 1e-9).sum()), rel.max())
        suspect |= rel > 1e-11
        suspect |= (runs[name][2] & bspl.Q_FALLBACK) != 0
    rng = np.random.default_rng(17)
    must = np.where(suspect)[0]
    rest = np.setdiff1d(np.arange(len(dp)), must)
    if len(must) > 80_000:
        must = rng.choice(must, 80_000, replace=False)
    pick = np.concatenate([must, rng.choice(rest, 20_000, replace=False)])
    print(f"oracle subset: {len(pick)} queries, {len(must)} of them where a fast path differs by more than "
          f"1e-11 x diag or used its FP64 fallback")
    qn = q.cpu().numpy()[pick]
    _, d_o = O.project_surfaces(ss, sq.proj_surf[pick], qn)
    err = np.abs(runs["plain"][1][pick] - d_o) / dp[pick]
    assert np.all(err <= 1e-9), (int((err > 1e-9).sum()), err.max())
    # the plain path's (u, v) reproduces its distance on the original surface
    S = O.eval_surfaces(ss, sq.proj_surf[pick], runs["plain"][0][pick])[0]
    assert np.all(np.abs(np.linalg.norm(S - qn, axis=1) - runs["plain"][1][pick]) <= 1e-9 * dp[pick])
