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
    lib.hd_surface_span.argtypes = [ctypes.c_int, ctypes.c_int, D, ctypes.c_int, D, ctypes.c_int, D, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, D, D, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int)]
    lib.hd_surface_span.restype = ctypes.c_int64
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
                k = hd.hd_surface_span(pu, pv, dp(U), qu, dp(V), qv, dp(P), nv, tol, diag, dp(ctrl), dp(pr), cap,
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
