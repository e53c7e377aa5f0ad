"""CPU check of the surface decomposition the GPU runs (csrc/decompose.cu,
compiled for the host span pair by span pair) against the oracle, bit for
bit: patch counts, bicubic nets and parameter boxes.  Surfaces of the
random-surface recipe, including nets whose span pairs are far longer in
one parameter than the other (where the split direction matters)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_11498_gb300 import synth
from paper_2504_11498_gb300.bspl import SREC32

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def hd(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hd") / "libhd.so")
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off", "-shared",
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_decompose.cu"),
           os.path.join(ROOT, "paper_2504_11498_gb300", "csrc", "scan.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    D = ctypes.POINTER(ctypes.c_double)
    lib.hd_box_diag.argtypes = [D, ctypes.c_int64]
    lib.hd_box_diag.restype = ctypes.c_double
    lib.hd_surface_span.argtypes = [ctypes.c_int, ctypes.c_int, D, ctypes.c_int, ctypes.c_int, D, ctypes.c_int, D,
                                    ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, D, D, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int)]
    lib.hd_surface_span.restype = ctypes.c_int64
    lib.hd_curve_span.argtypes = [ctypes.c_int, D, ctypes.c_int, D, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                  D, D, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    lib.hd_curve_span.restype = ctypes.c_int64
    return lib


def dp(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def host_decompose(hd, ss, tol):
    ctrl_all, pr_all, offs = [], [], [0]
    for s in range(ss.n):
        pu, pv, nu, nv = int(ss.deg_u[s]), int(ss.deg_v[s]), int(ss.n_u[s]), int(ss.n_v[s])
        U = np.ascontiguousarray(ss.knots_u[ss.knot_u_off[s]:ss.knot_u_off[s + 1]])
        V = np.ascontiguousarray(ss.knots_v[ss.knot_v_off[s]:ss.knot_v_off[s + 1]])
        P = np.ascontiguousarray(ss.cps[ss.cp_off[s]:ss.cp_off[s + 1]])
        diag = hd.hd_box_diag(dp(P), len(P))
        n = 0
        for a in range(nu):
            for b in range(nv):
                qu, qv = pu + a, pv + b
                if qu > nu - 1 or qv > nv - 1 or not (U[qu] < U[qu + 1]) or not (V[qv] < V[qv + 1]):
                    continue
                cap = 1 << 17
                ctrl = np.zeros((cap, 48))
                pr = np.zeros((cap, 4))
                err = ctypes.c_int()
                k = hd.hd_surface_span(pu, pv, dp(U), nu, qu, dp(V), qv, dp(P), nv, tol, diag, dp(ctrl), dp(pr), cap,
                                       ctypes.byref(err))
                assert 0 < k <= cap
                ctrl_all.append(ctrl[:k])
                pr_all.append(pr[:k])
                n += k
        offs.append(offs[-1] + n)
    return np.array(offs), np.concatenate(ctrl_all), np.concatenate(pr_all)


@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_surface_walk_bit_exact_with_oracle(hd, tol):
    ss, _ = synth.surface_set(seed=3, n_surf=12, n_proj=1, n_inv=1, n_range=(6, 12))
    if tol < 1e-5:  # the tight tolerance only where at most one direction is reduced
        ss = ss.subset([s for s in range(ss.n) if not (ss.deg_u[s] > 3 and ss.deg_v[s] > 3)])
    off, ctrl, pr = host_decompose(hd, ss, tol)
    ref = O.decompose_surfaces(ss, tol)
    assert np.array_equal(off, ref.seg_off)
    assert np.array_equal(pr, ref.prange)
    assert np.array_equal(ctrl.reshape(ref.ctrl.shape), ref.ctrl)


def test_anisotropic_span_pairs_stay_small(hd):
    """Surfaces of the 1,024-surface set with span pairs whose parameter
    lengths differ by four orders of magnitude: every span pair meets the
    tolerance well before the leaf cap, and host walk and oracle agree."""
    ss, _ = synth.surface_set(seed=3, n_surf=1024, n_proj=1, n_inv=1)
    sub = ss.subset([557, 81])
    off, ctrl, pr = host_decompose(hd, sub, 1e-4)
    ref = O.decompose_surfaces(sub, 1e-4)
    assert ref.status == 0
    assert np.array_equal(off, ref.seg_off) and np.array_equal(pr, ref.prange)
    assert np.array_equal(ctrl.reshape(ref.ctrl.shape), ref.ctrl)
    assert off[-1] < 20000


def test_patch_derivative_bounds_and_edge_flags(hd):
    """The certification search of the surface queries rests on the bounds
    the filling walk stores with each patch (FP32 record entries 56..61):
    |S_s|, |S_t|, |S_ss|, |S_st|, |S_tt| (and the third partials, entries
    62..65) of the ORIGINAL surface over the patch, in the patch's own
    parameters, and the edges across which the surface is C1.  Checked against the oracle's derivatives (Cox-de Boor,
    sampled on a 17 x 17 grid inside every patch), and the flags against the
    knot multiplicities, on surfaces with C0 creases and repeated knots."""
    hd.hd_surface_records.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    hd.hd_surface_records.restype = ctypes.c_int64
    rng = np.random.default_rng(41)
    pus, pvs, KU, KV, nets = [], [], [], [], []
    for pu, pv, nu, nv in ((3, 2, 7, 6), (5, 4, 9, 8), (2, 3, 6, 7), (4, 4, 8, 8)):
        U = synth.random_clamped_knots(rng, pu, nu, 0.3)  # repeated knots, creases where multiplicity = degree
        V = synth.random_clamped_knots(rng, pv, nv, 0.3)
        pus.append(pu)
        pvs.append(pv)
        KU.append(U)
        KV.append(V)
        nets.append(synth._sinusoid_net(rng, nu, nv))
    ss = synth.pack_surfaces(pus, pvs, KU, KV, nets)
    # strictly inside the patch: on a knot line the evaluator takes the next
    # span, whose derivatives differ at a crease
    g = np.concatenate([[1e-10], (np.arange(15) + 0.5) / 15, [1 - 1e-10]])
    checked = 0
    for s in range(ss.n):
        pu, pv, nu, nv = int(ss.deg_u[s]), int(ss.deg_v[s]), int(ss.n_u[s]), int(ss.n_v[s])
        U = np.ascontiguousarray(ss.knots_u[ss.knot_u_off[s]:ss.knot_u_off[s + 1]])
        V = np.ascontiguousarray(ss.knots_v[ss.knot_v_off[s]:ss.knot_v_off[s + 1]])
        P = np.ascontiguousarray(ss.cps[ss.cp_off[s]:ss.cp_off[s + 1]])
        diag = hd.hd_box_diag(dp(P), len(P))

        def smooth(K, p, n, x):
            return bool(K[p] < x < K[n] and np.sum(K == x) < p)

        for qu in range(pu, nu):
            for qv in range(pv, nv):
                if not (U[qu] < U[qu + 1] and V[qv] < V[qv + 1]):
                    continue
                cap = 4096
                rec = np.zeros((cap, SREC32), np.float32)
                pb = np.zeros((cap, 4))
                err = ctypes.c_int()
                k = hd.hd_surface_records(pu, pv, dp(U), nu, qu, dp(V), qv, dp(P), nv, 1e-3, diag,
                                          rec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), dp(pb), cap,
                                          ctypes.byref(err))
                assert 0 < k <= cap
                for j in range(k):
                    a0 = U[qu] + pb[j, 0] * (U[qu + 1] - U[qu])
                    a1 = U[qu] + pb[j, 1] * (U[qu + 1] - U[qu])
                    b0 = V[qv] + pb[j, 2] * (V[qv + 1] - V[qv])
                    b1 = V[qv] + pb[j, 3] * (V[qv + 1] - V[qv])
                    uu, vv = np.meshgrid(a0 + g * (a1 - a0), b0 + g * (b1 - b0), indexing="ij")
                    uv = np.stack([uu.ravel(), vv.ravel()], 1)
                    _, Su, Sv, Suu, Suv, Svv = O.eval_surfaces(ss, np.full(len(uv), s, np.int32), uv)
                    wu, wv = a1 - a0, b1 - b0  # d/ds = wu d/du
                    got = [np.linalg.norm(x, axis=1).max() for x in (Su * wu, Sv * wv, Suu * wu * wu,
                                                                     Suv * wu * wv, Svv * wv * wv)]
                    for m, bound in zip(got, rec[j, 56:61]):
                        assert m <= bound * (1 + 1e-6) + 1e-12, (s, qu, qv, j, m, bound)
                    # the bound is not loose beyond the convex-hull factor on these nets
                    assert rec[j, 56] <= 4 * got[0] + 1e-9
                    # third partials by central differences of the oracle's second
                    # partials (inner samples; relative error ~1e-8)
                    if j % 3 == 0:
                        inner = uv[(uv[:, 0] > a0 + 0.05 * wu) & (uv[:, 0] < a1 - 0.05 * wu) &
                                   (uv[:, 1] > b0 + 0.05 * wv) & (uv[:, 1] < b1 - 0.05 * wv)]
                        hu, hv = 1e-5 * wu, 1e-5 * wv
                        idx = np.full(len(inner), s, np.int32)
                        ev = lambda du_, dv_: O.eval_surfaces(ss, idx, inner + np.array([du_, dv_]))
                        up, um, vp, vm = ev(hu, 0), ev(-hu, 0), ev(0, hv), ev(0, -hv)
                        t3 = [(up[3] - um[3]) / (2 * hu) * wu ** 3, (vp[3] - vm[3]) / (2 * hv) * wu * wu * wv,
                              (up[5] - um[5]) / (2 * hu) * wu * wv * wv, (vp[5] - vm[5]) / (2 * hv) * wv ** 3]
                        for fd, bound in zip(t3, rec[j, 62:66]):
                            m3 = np.linalg.norm(fd, axis=1).max()
                            assert m3 <= bound * (1 + 1e-4) + 1e-9, (s, qu, qv, j, m3, bound)
                    f = int(rec[j, 61])
                    assert bool(f & 1) == (pb[j, 0] > 0 or smooth(U, pu, nu, U[qu]))
                    assert bool(f & 2) == (pb[j, 1] < 1 or smooth(U, pu, nu, U[qu + 1]))
                    assert bool(f & 4) == (pb[j, 2] > 0 or smooth(V, pv, nv, V[qv]))
                    assert bool(f & 8) == (pb[j, 3] < 1 or smooth(V, pv, nv, V[qv + 1]))
                    checked += 1
    assert checked > 50


def host_decompose_curves(hd, cs, tol):
    """The device's curve walk run on the host span by span (rational curves
    through the rational walk): seg_off, ctrl, prange."""
    ctrl_all, pr_all, offs = [], [], [0]
    for c in range(cs.n):
        p, U, P = cs.curve(c)
        U, P = np.ascontiguousarray(U), np.ascontiguousarray(P)
        w = cs.curve_weights(c)
        rat = w is not None and np.any(w != w[0])
        wa = np.ascontiguousarray(w) if rat else None
        diag = hd.hd_box_diag(dp(P), len(P))
        n = 0
        for q in range(p, len(P)):
            if not U[q] < U[q + 1]:
                continue
            cap = 1 << 16
            ctrl = np.zeros((cap, 12))
            pr = np.zeros((cap, 2))
            err = ctypes.c_int()
            k = hd.hd_curve_span(p, dp(U), q, dp(P), None if wa is None else wa.ctypes.data, tol, diag, dp(ctrl),
                                 dp(pr), cap, ctypes.byref(err))
            assert 0 < k <= cap and err.value == 0
            ctrl_all.append(ctrl[:k])
            pr_all.append(pr[:k])
            n += k
        offs.append(offs[-1] + n)
    return np.array(offs), np.concatenate(ctrl_all).reshape(-1, 4, 3), np.concatenate(pr_all)


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-11])
def test_rational_curve_walk_bit_exact(hd, tol):
    """The rational walk (homogeneous pieces, Hermite cubics, certified
    bound) agrees with the oracle bit for bit, on random NURBS with weights
    over a 16:1 range and on exact circles."""
    cs, _ = synth.nurbs_curve_set(seed=31, n_curves=24, n_proj=1, n_inv=0, ncp_range=(8, 20), w_range=(0.25, 4.0))
    circ = synth.nurbs_circles(seed=32, n_curves=4, n_proj=1)[0]
    for s in (cs, circ):
        offs, ctrl, pr = host_decompose_curves(hd, s, tol)
        ref = O.decompose_curves(s, tol)
        assert np.array_equal(offs, ref.seg_off)
        assert np.array_equal(ctrl, ref.ctrl)
        assert np.array_equal(pr, ref.prange)


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_high_degree_curve_walk_bit_exact(hd, tol):
    """Every walk instance the device launches (degrees 1..7 by the matrix
    route, 8..15 and 16..31 by the blossom with the coefficient tables,
    32..63 by the blossom with the coefficients computed inline),
    non-rational and rational: the walk agrees with the oracle bit for
    bit."""
    rng = np.random.default_rng(44)
    degs, knots, cps, ws = [], [], [], []
    for p in (5, 7, 8, 12, 15, 16, 31, 32, 40, 51, 63):
        ncp = p + int(rng.integers(1, 6))
        degs.append(p)
        knots.append(synth.random_clamped_knots(rng, p, ncp))
        cps.append(rng.uniform(0.0, 1.0, size=(ncp, 3)))
        ws.append(np.exp(rng.uniform(np.log(0.5), np.log(2.0), ncp)))
    for s in (synth.pack_curves(degs, knots, cps), synth.pack_curves(degs, knots, cps, ws)):
        offs, ctrl, pr = host_decompose_curves(hd, s, tol)
        ref = O.decompose_curves(s, tol)
        assert np.array_equal(offs, ref.seg_off)
        assert np.array_equal(ctrl, ref.ctrl)
        assert np.array_equal(pr, ref.prange)
