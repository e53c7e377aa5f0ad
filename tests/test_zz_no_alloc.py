"""The scratch-free projection entry point.

Some callers cannot allocate GPU memory for the library's workspace (their
application owns every byte of device memory through its own pool, they run
inside a plugin or callback that must not call the CUDA allocator, or they
cannot afford the synchronisation an allocation brings).  For them
bspl_project_curves_noalloc keeps its scratch in a fixed array inside the
library.  This file checks, through the C ABI, that it answers exactly like
bspl_project_curves on two calls in a row (the second call reuses the
scratch the first one left behind), and that it refuses batches larger than
its fixed limit.  It is meant to run last (and also works on its own).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_on_two_calls():
    from oracle import oracle as O
    from paper_2504_11498_gb300 import build, bspl, synth
    build.build()
    dev = "cuda"
    cs, qs = synth.curve_set(seed=7, n_curves=512, n_proj=300_000, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, dev), 1e-10)
    qc = torch.as_tensor(qs.proj_curve, device=dev)
    q = torch.as_tensor(qs.proj_xyz, device=dev)
    diag = O.curve_diag(cs)[qs.proj_curve]
    for prec in (bspl.FP64, bspl.MIXED):
        opts = bspl.make_options(prec=prec)
        ref = bspl.bspl_project_curves(segs, qc, q, opts)
        torch.cuda.synchronize()
        t_ref, d_ref = ref.param.cpu().numpy().copy(), ref.dist.cpu().numpy().copy()
        for call in range(2):
            r = bspl.bspl_project_curves_noalloc(segs, qc, q, opts)
            torch.cuda.synchronize()
            d = r.dist.cpu().numpy()
            t = r.param.cpu().numpy()
            assert np.all(np.abs(d - d_ref) <= 1e-12 * diag), (prec, call)
            assert np.array_equal(r.status.cpu().numpy(), ref.status.cpu().numpy())
            assert np.all(np.isfinite(t))


def test_noalloc_rejects_batches_over_its_limit():
    from paper_2504_11498_gb300 import build, bspl, synth
    build.build()
    dev = "cuda"
    cs, _ = synth.single_cubic(n_proj=1, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, dev), 0.0)
    n = bspl.NOALLOC_MAX_QUERIES + 1
    qc = torch.zeros(n, dtype=torch.int32, device=dev)
    q = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    with pytest.raises(bspl.BsplError, match="ENOSPACE"):
        bspl.bspl_project_curves_noalloc(segs, qc, q)


def test_noalloc_learned_precision_within_and_over_its_limit():
    """The learned precision also keeps its candidate and pair buffers in
    the fixed array, about 1.4 KB per query: a batch that fits answers like the
    regular entry point (two calls in a row), a larger one is refused with
    ENOSPACE rather than mistaken for a caller error."""
    from oracle import oracle as O
    from paper_2504_11498_gb300 import build, bspl, synth
    build.build()
    dev = "cuda"
    cs, qs = synth.curve_set(seed=7, n_curves=512, n_proj=40_000, n_inv=1)
    segs = bspl.decompose(bspl.DeviceCurves(cs, dev), 1e-10)
    limit = bspl.SCRATCH_BYTES
    n_fit = 4000
    assert bspl.workspace_bytes(bspl.OP_QUERY_CURVES_LEARNED, segs.n, 0, 0, n_fit) <= limit
    assert bspl.workspace_bytes(bspl.OP_QUERY_CURVES_LEARNED, segs.n, 0, 0, 40_000) > limit
    mlp = bspl.Mlp(synth.mlp_init(7), dev)
    opts = bspl.make_options(prec=bspl.LEARNED_MIXED, mlp=mlp)
    qc = torch.as_tensor(qs.proj_curve[:n_fit], device=dev)
    q = torch.as_tensor(qs.proj_xyz[:n_fit], device=dev)
    diag = O.curve_diag(cs)[qs.proj_curve[:n_fit]]
    ref = bspl.bspl_project_curves(segs, qc, q, opts)
    torch.cuda.synchronize()
    d_ref, st_ref = ref.dist.cpu().numpy().copy(), ref.status.cpu().numpy().copy()
    for call in range(2):
        r = bspl.bspl_project_curves_noalloc(segs, qc, q, opts)
        torch.cuda.synchronize()
        assert np.all(np.abs(r.dist.cpu().numpy() - d_ref) <= 1e-12 * diag), call
        assert np.array_equal(r.status.cpu().numpy(), st_ref)
    qc = torch.as_tensor(qs.proj_curve, device=dev)
    q = torch.as_tensor(qs.proj_xyz, device=dev)
    with pytest.raises(bspl.BsplError, match="ENOSPACE"):
        bspl.bspl_project_curves_noalloc(segs, qc, q, opts)
