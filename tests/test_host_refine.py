"""CPU check of the refinement the GPU runs on the original curves
(csrc/eval.cu, compiled for the host) against the oracle, at every degree
class (1..7, 8..31, 32..63), non-rational and rational:

* its evaluation of C, C', C'' against the oracle's;
* the whole query path emulated: the minimum of the decomposed cubics (the
  oracle's decomposition, searched here by sampling and Newton on the cubic,
  as the query kernels do), then the refinement from it, within 1e-9 x diag
  of the oracle's projection on every query;
* from those starts, the refinement converges in about two evaluations and
  never ends farther than it started (beyond rounding).  At degrees 8 and above the
  cubics come from the blossom extraction; with the matrix route the
  degree-31 curve's cubics were off by about 1e-2 of the control points'
  size and a query's refined distance by 2.8e-3 x diag.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_11498_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def hr(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hr") / "libhr.so")
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "host_refine.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.hr_eval.argtypes = [ctypes.c_int, D, ctypes.c_int, D, ctypes.c_void_p, ctypes.c_double, D, D, D]
    lib.hr_refine.argtypes = [ctypes.c_int, D, ctypes.c_int, D, ctypes.c_void_p, D, ctypes.c_int, D, D,
                              ctypes.POINTER(ctypes.c_int)]
    lib.hr_refine.restype = ctypes.c_int
    return lib


def dp(x):
    return x.ctypes.data_as(D)


def high_set(rational, seed=52, degrees=(3, 31, 32, 40, 51, 63)):
    """The curve set of the GPU high-degree test (same draws)."""
    rng = np.random.default_rng(seed)
    degs, knots, cps, ws = [], [], [], []
    for p in degrees:
        ncp = p + int(rng.integers(1, 8))
        degs.append(p)
        knots.append(synth.random_clamped_knots(rng, p, ncp))
        cps.append(rng.uniform(0.0, 1.0, size=(ncp, 3)))
        ws.append(np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncp)))
    return synth.pack_curves(degs, knots, cps, ws if rational else None)


def curve_arrays(cs, c):
    p, U, P = cs.curve(c)
    w = cs.curve_weights(c)
    return (p, np.ascontiguousarray(U), np.ascontiguousarray(P),
            None if w is None else np.ascontiguousarray(w))


@pytest.mark.parametrize("rational", [False, True])
def test_refinement_evaluation_matches_oracle(hr, rational):
    cs = high_set(rational, degrees=(3, 7, 10, 31, 32, 40, 51, 63))
    t = np.linspace(0.0, 1.0, 97)
    for c in range(cs.n):
        p, U, P, w = curve_arrays(cs, c)
        ref = O.eval_curves(cs, np.full(len(t), c, np.int32), t)
        got = np.zeros((3, len(t), 3))
        for k, tk in enumerate(t):
            a, b, d = np.zeros(3), np.zeros(3), np.zeros(3)
            hr.hr_eval(p, dp(U), len(P) - 1, dp(P), None if w is None else w.ctypes.data, tk, dp(a), dp(b), dp(d))
            got[:, k] = a, b, d
        for i in range(3):
            scale = 1.0 + np.abs(ref[i]).max()
            assert np.abs(got[i] - ref[i]).max() <= 1e-13 * scale, (p, i)


def cubic_minimum(R, q):
    """(u, D) minimising |R(u) - q|^2 over [0, 1] for the cubic Bezier R:
    the best of 65 samples, then safeguarded Newton on E = (R - q).R'."""
    u = np.linspace(0.0, 1.0, 65)
    B = np.stack([math.comb(3, i) * u ** i * (1 - u) ** (3 - i) for i in range(4)], 1)
    d2 = ((B @ R - q) ** 2).sum(1)
    k = int(d2.argmin())
    lo, hi, x = u[max(k - 1, 0)], u[min(k + 1, 64)], u[k]
    a = [R[1] - R[0], R[2] - R[1], R[3] - R[2]]
    for _ in range(60):
        b = np.array([(1 - x) ** 3, 3 * x * (1 - x) ** 2, 3 * x * x * (1 - x), x ** 3])
        C = b @ R
        C1 = 3 * ((1 - x) ** 2 * a[0] + 2 * x * (1 - x) * a[1] + x * x * a[2])
        C2 = 6 * ((1 - x) * (a[1] - a[0]) + x * (a[2] - a[1]))
        E, Ep = (C - q) @ C1, C1 @ C1 + (C - q) @ C2
        xn = x - E / Ep if Ep > 0 else 0.5 * (lo + hi)
        if E > 0:
            hi = x
        elif E < 0:
            lo = x
        if not lo <= xn <= hi:
            xn = 0.5 * (lo + hi)
        if abs(xn - x) <= 1e-16:
            break
        x = xn
    b = np.array([(1 - x) ** 3, 3 * x * (1 - x) ** 2, 3 * x * x * (1 - x), x ** 3])
    return x, float(((b @ R - q) ** 2).sum())


@pytest.mark.parametrize("rational", [False, True])
def test_query_path_emulated_then_refined_matches_oracle(hr, rational):
    tol = 1e-9
    cs = high_set(rational)
    rng = np.random.default_rng(53)
    rng.uniform(0.0, 1.0, 3000)  # the GPU test's inversion parameters
    qc = np.repeat(np.arange(cs.n, dtype=np.int32), 500)
    lo, hi = synth.cp_boxes(cs)
    q = synth._box_queries(rng, lo, hi, qc, scale=1.3)
    pick = np.concatenate([np.where(qc == c)[0][:120] for c in range(cs.n)])
    if not rational:
        pick = np.union1d(pick, [524])  # the query the matrix route's degree-31 cubics sent astray
    _, d_o = O.project_curves(cs, qc[pick], q[pick])
    dec = O.decompose_curves(cs, tol)
    diag = O.curve_diag(cs)
    u = np.linspace(0.0, 1.0, 33)
    B = np.stack([math.comb(3, i) * u ** i * (1 - u) ** (3 - i) for i in range(4)], 1)
    worst = 0.0
    for n, k in enumerate(pick):
        c = int(qc[k])
        p, U, P, w = curve_arrays(cs, c)
        s0, s1 = dec.seg_off[c], dec.seg_off[c + 1]
        # the candidate segments: the best sampled ones (the approximant's
        # global minimum lies in one of them)
        pts = np.einsum("ui,sic->suc", B, dec.ctrl[s0:s1])
        dmin = ((pts - q[k]) ** 2).sum(2).min(1)
        best = (np.inf, 0.0)
        for s in np.argsort(dmin)[:4]:
            x, d2 = cubic_minimum(dec.ctrl[s0 + s], q[k])
            if d2 < best[0]:
                t0, t1 = dec.prange[s0 + s]
                best = (d2, t0 + x * (t1 - t0))
        t = ctypes.c_double(best[1])
        Dv, nev = ctypes.c_double(), ctypes.c_int()
        qq = np.ascontiguousarray(q[k])
        hr.hr_refine(p, dp(U), len(P) - 1, dp(P), None if w is None else w.ctypes.data, dp(qq), 16,
                     ctypes.byref(t), ctypes.byref(Dv), ctypes.byref(nev))
        err = abs(math.sqrt(Dv.value) - d_o[n]) / diag[c]
        worst = max(worst, err)
        assert err <= 1e-9, (c, p, int(k), err, t.value)
    assert worst <= 1e-9


def test_refinement_settles_in_about_two_evaluations(hr):
    """From the query path's answer (emulated as above) on the curve-set
    recipe, non-rational and rational, projections and inversions: the
    refinement converges, taking about two evaluations per query (the start
    and one Newton step, whose change of D is within D's rounding), and
    never ends farther than its start beyond that rounding."""
    for make in (synth.curve_set, synth.nurbs_curve_set):
        cs, qs = make(seed=61, n_curves=24, n_proj=300, n_inv=300, ncp_range=(8, 20))
        dec = O.decompose_curves(cs, 1e-10)
        inv_pts = O.eval_curves(cs, qs.inv_curve, qs.inv_t)[0]
        qc = np.concatenate([qs.proj_curve, qs.inv_curve])
        q = np.concatenate([qs.proj_xyz, inv_pts])
        evals, conv = [], []
        u = np.linspace(0.0, 1.0, 33)
        B = np.stack([math.comb(3, i) * u ** i * (1 - u) ** (3 - i) for i in range(4)], 1)
        for k in range(len(qc)):
            c = int(qc[k])
            p, U, P, w = curve_arrays(cs, c)
            s0, s1 = dec.seg_off[c], dec.seg_off[c + 1]
            pts = np.einsum("ui,sic->suc", B, dec.ctrl[s0:s1])
            dmin = ((pts - q[k]) ** 2).sum(2).min(1)
            best = (np.inf, 0.0)
            for s in np.argsort(dmin)[:4]:
                x, d2 = cubic_minimum(dec.ctrl[s0 + s], q[k])
                if d2 < best[0]:
                    t0, t1 = dec.prange[s0 + s]
                    best = (d2, t0 + x * (t1 - t0))
            t = ctypes.c_double(best[1])
            Dv, nev = ctypes.c_double(), ctypes.c_int()
            qq = np.ascontiguousarray(q[k])
            C0 = O.eval_curves(cs, np.array([c], np.int32), np.array([best[1]]))[0][0]
            d_start = np.linalg.norm(C0 - q[k])
            ok = hr.hr_refine(p, dp(U), len(P) - 1, dp(P), None if w is None else w.ctypes.data, dp(qq), 16,
                              ctypes.byref(t), ctypes.byref(Dv), ctypes.byref(nev))
            assert math.sqrt(Dv.value) <= d_start + 1e-14 * (1 + d_start)
            evals.append(nev.value)
            conv.append(ok)
        assert all(conv)
        assert np.mean(evals) <= 2.3 and max(evals) <= 14, (make.__name__, np.mean(evals), max(evals))


def test_refinement_reaches_minima_at_c0_joints(hr):
    """Starts a short way (1e-9 and 1e-6 of the domain, either side) from
    minima that lie on or next to a C0 joint (a knot of full multiplicity,
    where D has a kink): the refinement reaches them.  (The full Newton step
    from the far side of the joint overshoots it; the knot it crossed is
    tried as well.)"""
    cs = high_set(False)
    p, U, P, w = curve_arrays(cs, 0)  # the cubic with a triple interior knot
    inner, counts = np.unique(U[p + 1:len(P)], return_counts=True)
    joints = inner[counts >= p]
    assert len(joints) >= 1
    rng = np.random.default_rng(53)
    rng.uniform(0.0, 1.0, 3000)
    qc = np.repeat(np.arange(cs.n, dtype=np.int32), 500)
    lo, hi = synth.cp_boxes(cs)
    q = synth._box_queries(rng, lo, hi, qc, scale=1.3)
    sel = np.where(qc == 0)[0]
    t_o, d_o = O.project_curves(cs, qc[sel], q[sel])
    near = np.min(np.abs(t_o[:, None] - joints[None, :]), axis=1) <= 1e-5
    assert near.sum() >= 5
    diag = O.curve_diag(cs)[0]
    for k in np.where(near)[0]:
        qq = np.ascontiguousarray(q[sel[k]])
        for off in (-1e-6, -1e-9, 1e-9, 1e-6):
            t = ctypes.c_double(min(max(t_o[k] + off, U[p]), U[len(P)]))
            Dv, nev = ctypes.c_double(), ctypes.c_int()
            hr.hr_refine(p, dp(U), len(P) - 1, dp(P), None, dp(qq), 16, ctypes.byref(t), ctypes.byref(Dv),
                         ctypes.byref(nev))
            err = abs(math.sqrt(Dv.value) - d_o[k]) / diag
            assert err <= 1e-9, (int(k), off, err, t.value, t_o[k])
