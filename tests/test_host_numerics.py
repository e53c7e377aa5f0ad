"""CPU tests of the curve query numerics shared with the GPU kernels
(csrc/query_common.cuh compiled for the host): decisions of the certified
isolation and of the two FP64 Newton steps on constructed segments whose
critical values are exact in FP32 and FP64."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def hn(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hn") / "libhn.so")
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "host_numerics.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    F = ctypes.POINTER(ctypes.c_float)
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.hn_bernstein_f.argtypes = [F, F]
    lib.hn_end_signs_d.argtypes = [D, I, I]
    lib.hn_classify.argtypes = [F]
    lib.hn_isolate_f.argtypes = [F, ctypes.c_int, F, I, F]
    lib.hn_isolate_f.restype = ctypes.c_float
    lib.hn_isolate_d.argtypes = [D, D, ctypes.c_int]
    lib.hn_isolate_d.restype = ctypes.c_double
    lib.hn_finish64.argtypes = [D, D, D, D]
    lib.hn_finish64.restype = ctypes.c_double
    lib.hn_quartic_d.argtypes = [D, D]
    lib.hn_quartic_f.argtypes = [F, F]
    lib.hn_clip_f.argtypes = [F, ctypes.c_float, ctypes.c_int, F, I, I]
    lib.hn_clip_f.restype = ctypes.c_float
    return lib


def fp(x):
    return np.ascontiguousarray(x, np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def dp(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# C(u) - q = (u - 1, 1 - 4u + 8u^2 - 4u^3, 0): at u = 1 the point is (0, 1, 0)
# and the tangent (1, 0, 0), so E(1) = 0 exactly in any precision, and u = 1
# is a local maximum of D (D''(1) < 0); E has three roots, the minimum is
# interior.
HOOK = np.array([-1.0, 1.0, 0.0, 1.0, -4.0, 0.0, 0.0, 8.0, 0.0, 0.0, -4.0, 0.0])
# C(u) - q = (1 - (1-u)^3 - 1/2, 1, 0): E = x x' = 3 (1-u)^2 (x) has one
# crossing from - to + (the minimum, at 1 - 2^(-1/3)) and a double root at
# u = 1, where D flattens out; its last Bernstein coefficients are exactly 0.
FLAT = np.array([-0.5, 1.0, 0.0, 3.0, 0.0, 0.0, -3.0, 0.0, 0.0, 1.0, 0.0, 0.0])


def d2(a, u):
    u = np.asarray(u, float)[..., None]
    return np.sum((a[0:3] + u * (a[3:6] + u * (a[6:9] + u * a[9:12]))) ** 2, axis=-1)


def argmin_dense(a):
    us = np.linspace(0, 1, 400001)
    return us[np.argmin(d2(a, us))]


def isolate32(hn, a, btol=None):
    unc = ctypes.c_int()
    sec = np.zeros(3, np.float32)
    u = hn.hn_isolate_f(fp(a), 16, fp(btol) if btol is not None else None, ctypes.byref(unc),
                        sec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return u, unc.value


def finish(hn, a, u0):
    u, last = ctypes.c_double(u0), ctypes.c_double()
    D = hn.hn_finish64(dp(np.array(a, float)), dp(np.zeros(3)), ctypes.byref(u), ctypes.byref(last))
    return u.value, last.value, D


def test_end_signs_skip_zeros(hn):
    f, l = ctypes.c_int(), ctypes.c_int()
    for b, want in (([-1, -2, -1, 2, 1, 0], (-1, 1)), ([0, 0, 3, -1, 0, 0], (1, -1)), ([0] * 6, (0, 0)),
                    ([-1, 0, 0, 0, 0, 2], (-1, 1))):
        hn.hn_end_signs_d(dp(np.array(b, float)), ctypes.byref(f), ctypes.byref(l))
        assert (f.value, l.value) == want


def test_flat_end_has_exact_zero_end_coefficient(hn):
    b = np.zeros(6, np.float32)
    v = hn.hn_bernstein_f(fp(FLAT), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    assert b[5] == 0.0 and b[0] < 0 and v in (1, 2)
    assert abs(argmin_dense(FLAT) - (1 - 2 ** (-1 / 3))) < 1e-5


@pytest.mark.parametrize("a", [HOOK, FLAT], ids=["three-changes", "zero-end"])
def test_isolation_finds_the_interior_minimum(hn, a):
    u_star = argmin_dense(a)
    assert 0.05 < u_star < 0.95 and d2(a, u_star) < min(d2(a, 0.0), d2(a, 1.0))
    for btol in (None, np.full(6, 1e-6, np.float32)):
        u, _ = isolate32(hn, a, btol)
        assert abs(u - u_star) < 1e-4, u
    u = hn.hn_isolate_d(dp(np.array(a, float)), dp(np.zeros(3)), 30)
    assert abs(u - u_star) < 1e-5


@pytest.mark.parametrize("a", [HOOK, FLAT], ids=["three-changes", "zero-end"])
def test_fp64_steps_do_not_converge_at_a_flat_end(hn, a):
    # E(1) = 0 and E'(1) <= 0: no Newton step; u = 1 is not a minimum
    _, last, _ = finish(hn, a, 1.0)
    assert last > 1e-9
    # from the FP32 isolation's minimiser the steps converge to the minimum
    u_star = argmin_dense(a)
    u32, _ = isolate32(hn, a)
    u, last, _ = finish(hn, a, float(u32))
    assert last <= 1e-9 and abs(u - u_star) < 1e-5


def test_fp64_steps_converge_at_a_valid_end(hn):
    # a straight segment moving away from q: the minimum is at u = 0 (E(0) > 0)
    a = np.array([1.0, 0, 0, 1.0, 0, 0, 0, 0, 0, 0, 0, 0])
    u, last, D = finish(hn, a, 0.0)
    assert last <= 1e-9 and u == 0.0 and D == 1.0
    # and one moving towards q ending short of it: the minimum is at u = 1 (E(1) < 0)
    a = np.array([-3.0, 0, 0, 1.0, 0, 0, 0, 0, 0, 0, 0, 0])
    u, last, D = finish(hn, a, 1.0)
    assert last <= 1e-9 and u == 1.0 and D == 4.0


def cubic(x, y=(1.0, 0, 0, 0)):
    """local-frame coefficients of C(u) - q = (x(u), y(u), 0), power basis"""
    return np.array([x[0], y[0], 0, x[1], y[1], 0, x[2], y[2], 0, x[3], y[3], 0], float)


KINDS = {"seed": 0, "end0": 1, "end1": 2, "ends": 3, "iso": 4, "isou": 5}


@pytest.mark.parametrize("a,kind", [
    (cubic((-0.5, 1, 0, 0)), "seed"),        # passes q at u = 1/2: one change from - to +
    (cubic((1, 1, 0, 0)), "end0"),           # moves away from q
    (cubic((-2, 1, 0, 0)), "end1"),          # moves towards q, stops short
    (cubic((1, 1, -1, 0), (0, 0, 0, 0)), "ends"),  # x = 1 + u - u^2 > 0 peaks inside: + to -
    (FLAT, "isou"),                          # last coefficients exactly 0: uncertain at the end
    (cubic((-0.4, 1, 0, 0)), "seed"),        # b2 exactly 0 between - and +: one change either way
], ids=["seed", "end0", "end1", "ends", "flat-end", "lone-zero"])
def test_classification(hn, a, kind):
    assert hn.hn_classify(fp(a)) == KINDS[kind]


def test_classification_iso_certain(hn):
    # a random cubic whose E has three certified sign changes
    rng = np.random.default_rng(3)
    for _ in range(20000):
        a = rng.uniform(-1, 1, 12)
        b = np.zeros(6, np.float32)
        v = hn.hn_bernstein_f(fp(a), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if v >= 2 and np.min(np.abs(b)) > 1e-2 * np.max(np.abs(b)):
            assert hn.hn_classify(fp(a)) == KINDS["iso"]
            return
    pytest.fail("no cubic with certified changes found")


@pytest.mark.parametrize("btol,unsure", [
    ([0, 0, 0.2, 0, 0, 0], 0),    # b2 = -0.1 between -0.3 and +0.1: the count cannot change
    ([0, 0.4, 0, 0, 0, 0], 1),    # b1 = -0.3 between -0.5 and -0.1: could add two changes
    ([0, 0, 0.2, 0.2, 0, 0], 1),  # a run of two
    ([0.6, 0, 0, 0, 0, 0], 1),    # at an end
])
def test_uncertainty_only_where_it_matters(hn, btol, unsure):
    a = cubic((-0.5, 1, 0, 0))    # b = (-0.5, -0.3, -0.1, 0.1, 0.3, 0.5), one change
    _, unc = isolate32(hn, a, np.array(btol, np.float32))
    assert unc == unsure


# ------------------------------------------------ the paper's search stage

def quartic(hn, c, f32=False):
    x = np.zeros(4, np.float32 if f32 else np.float64)
    if f32:
        n = hn.hn_quartic_f(fp(c), x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    else:
        n = hn.hn_quartic_d(dp(np.array(c, float)), dp(x))
    return np.sort(x[:n].astype(np.float64))


def test_quartic_roots_closed_form_cases(hn):
    # four real roots, two real and a complex pair, biquadratic, cubic fallback
    assert np.allclose(quartic(hn, np.poly([0.9, 0.3, -1.2, 2.5])[::-1] * 3.0), [-1.2, 0.3, 0.9, 2.5], atol=1e-10)
    c = np.polymul(np.poly([0.25, 0.75]), [1.0, 0.4, 2.0])[::-1]  # x^2 + 0.4 x + 2 has no real root
    assert np.allclose(quartic(hn, c), [0.25, 0.75], atol=1e-12)
    assert np.allclose(quartic(hn, [4.0, 0.0, -5.0, 0.0, 1.0]), [-2, -1, 1, 2], atol=1e-12)
    assert np.allclose(quartic(hn, [6.0, -11.0, 6.0, -1.0, 0.0]), [1, 2, 3], atol=1e-9)  # -(x-1)(x-2)(x-3)
    assert len(quartic(hn, [1.0, 0.0, 1.0, 0.0, 1.0])) == 0  # x^4 + x^2 + 1 > 0


def test_quartic_roots_random_against_numpy(hn):
    rng = np.random.default_rng(41)
    for _ in range(2000):
        r = np.sort(rng.uniform(-2, 2, 4))
        if np.min(np.diff(r)) < 1e-2:
            continue
        c = (np.poly(r) * rng.uniform(0.5, 3) * rng.choice([-1, 1]))[::-1]
        got = quartic(hn, c)
        assert len(got) == 4 and np.allclose(got, r, atol=1e-8), (r, got)
        # FP32: every root in (0, 1) found to FP32-level accuracy
        g32 = quartic(hn, c, f32=True)
        for x in r[(r > 0) & (r < 1)]:
            assert np.min(np.abs(g32 - x)) < 2e-3, (r, g32)


def dense_min(a, n=50001):
    u = np.linspace(0, 1, n)
    D = d2(a, u)
    k = int(np.argmin(D))
    return u[k], D[k]


def test_clip_search_finds_the_global_minimum(hn):
    """Random local-frame cubics (q at the origin): the paper's search
    returns the global minimiser of D on [0, 1] to FP32 accuracy, as dense
    FP64 sampling finds it, and agrees with the certified isolation."""
    rng = np.random.default_rng(43)
    worst = 0.0
    for _ in range(1500):
        P = rng.uniform(-1, 1, (4, 3))
        # power coefficients of the Bezier cubic (component-wise), q = origin
        a = np.array([P[0], 3 * (P[1] - P[0]), 3 * (P[2] - 2 * P[1] + P[0]), P[3] - 3 * P[2] + 3 * P[1] - P[0]])
        a = a.reshape(-1)
        sec = np.zeros(3, np.float32)
        nmin, uns = ctypes.c_int(), ctypes.c_int()
        u = hn.hn_clip_f(fp(a), 1e-6, 12, sec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(nmin),
                         ctypes.byref(uns))
        _, Dm = dense_min(a)
        Du = float(d2(a, np.array([u]))[0])
        scale = np.sum(np.abs(a)) ** 2
        worst = max(worst, (Du - Dm) / scale)
        assert Du - Dm <= 2e-6 * scale, (P, u, Du, Dm)
        u_iso, _ = isolate32(hn, a)
        assert abs(Du - float(d2(a, np.array([u_iso]))[0])) <= 2e-6 * scale
    print(f"worst (D_clip - D_dense) / scale: {worst:.3g}")


def test_clip_search_certifies_most_pairs(hn):
    """The closed-form split leaves pieces whose Bernstein sign changes
    certify them (after at most three halvings) on all but a few percent of
    random pairs; the others are flagged for the FP64 decision."""
    rng = np.random.default_rng(5)
    unsure = 0
    n = 4000
    for _ in range(n):
        P = rng.uniform(-1, 1, (4, 3)) * rng.uniform(0.01, 1)
        q = rng.uniform(-0.75, 0.75, 3)
        a = np.array([P[0] - q, 3 * (P[1] - P[0]), 3 * (P[2] - 2 * P[1] + P[0]), P[3] - 3 * P[2] + 3 * P[1] - P[0]])
        c = np.abs(a)
        ea = sum(np.array([c[0, k] * c[1, k], 2 * c[0, k] * c[2, k] + c[1, k] ** 2,
                           3 * c[0, k] * c[3, k] + 3 * c[1, k] * c[2, k], 4 * c[1, k] * c[3, k] + 2 * c[2, k] ** 2,
                           5 * c[2, k] * c[3, k], 3 * c[3, k] ** 2]) for k in range(3))
        sec = np.zeros(3, np.float32)
        nmin, uns = ctypes.c_int(), ctypes.c_int()
        hn.hn_clip_f(fp(a.reshape(-1)), float(1e-5 * ea.sum()), 12, sec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                     ctypes.byref(nmin), ctypes.byref(uns))
        unsure += uns.value
    assert unsure < 0.03 * n, unsure
