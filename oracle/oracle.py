"""Python face of the CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Thin ctypes marshalling over ``bspl_oracle.c`` plus the paper's printed
matrices written out in NumPy (``tables`` below).  Only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it;
the GPU library never imports it and it never imports the GPU library.

Curve and surface sets are taken by duck typing (any object with the CSR
attributes ``degree, knot_off, knots, cp_off, cps`` for curves and
``deg_u, deg_v, n_u, n_v, knot_u_off, knots_u, knot_v_off, knots_v, cp_off,
cps`` for surfaces).
"""
from __future__ import annotations

import ctypes as C
import math
import threading

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")

OK, EINVAL, ENOSPACE, ENOTCONV = 0, 1, 2, 4


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_build.build())
            I64, I32, D = C.c_int64, C.c_int32, C.c_double
            vp = C.c_void_p
            L.orc_gram.restype = D
            L.orc_gram.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
            L.orc_basis.argtypes = [C.c_int, _f64p, I64, D, C.POINTER(C.c_int), _f64p]
            L.orc_eval_curves.argtypes = [I64, _i32p, _i64p, _f64p, _i64p, _f64p, vp, I64, _i32p, _f64p, _f64p]
            L.orc_eval_surfaces.argtypes = [I64, _i32p, _i32p, _i32p, _i32p, _i64p, _f64p, _i64p, _f64p,
                                            _i64p, _f64p, vp, I64, _i32p, _f64p, _f64p]
            L.orc_boehm_bezier.argtypes = [C.c_int, _f64p, I64, _f64p, I64, _f64p, I64, C.POINTER(I64)]
            L.orc_span_bezier.argtypes = [C.c_int, _f64p, I64, _f64p, I64, _f64p, I64, C.POINTER(I64)]
            L.orc_span_blossom.argtypes = [C.c_int, _f64p, I64, _f64p, I64, _f64p, I64, C.POINTER(I64)]
            L.orc_reduce_g1.argtypes = [C.c_int, _f64p, _f64p, _f64p, C.c_int]
            L.orc_to_cubic.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_bound2.restype = D
            L.orc_bound2.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_halve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
            L.orc_elevate.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_decompose_curves.argtypes = [I64, _i32p, _i64p, _f64p, _i64p, _f64p, vp, D, _i64p, I64, vp, vp,
                                               C.POINTER(I64), C.POINTER(C.c_int)]
            L.orc_decompose_surfaces.argtypes = [I64, _i32p, _i32p, _i32p, _i32p, _i64p, _f64p, _i64p, _f64p,
                                                 _i64p, _f64p, vp, D, _i64p, I64, vp, vp, C.POINTER(I64),
                                                 C.POINTER(C.c_int)]
            L.orc_rsurf_hermite.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
            L.orc_rsurf_bound2.restype = D
            L.orc_rsurf_bound2.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
            L.orc_project_curves.argtypes = [I64, _i32p, _i64p, _f64p, _i64p, _f64p, vp, I64, _i32p, _f64p,
                                             _f64p, _f64p, C.c_int]
            L.orc_rspan_bezier.argtypes = [C.c_int, _f64p, I64, _f64p, _f64p, I64, _f64p, I64, C.POINTER(I64)]
            L.orc_rhermite.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_rbound2.restype = D
            L.orc_rbound2.argtypes = [C.c_int, _f64p, _f64p]
            L.orc_rhalve.argtypes = [C.c_int, _f64p, _f64p, _f64p]
            L.orc_curve_deriv_bounds.argtypes = [C.c_int, _f64p, I64, _f64p, vp, C.c_int, C.POINTER(D),
                                                 C.POINTER(D)]
            L.orc_project_surfaces.argtypes = [I64, _i32p, _i32p, _i32p, _i32p, _i64p, _f64p, _i64p, _f64p,
                                               _i64p, _f64p, vp, I64, _i32p, _f64p, _f64p, _f64p, C.c_int]
            L.orc_surf_deriv_bounds.argtypes = [C.c_int, C.c_int, _f64p, C.c_int, _f64p, C.c_int, _f64p, vp,
                                                C.c_int, C.c_int, _f64p]
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _a(x, dt):
    return np.ascontiguousarray(np.asarray(x, dtype=dt))


def _curve_args(cs):
    return (int(len(cs.degree)), _a(cs.degree, np.int32), _a(cs.knot_off, np.int64), _a(cs.knots, np.float64),
            _a(cs.cp_off, np.int64), _a(cs.cps, np.float64).reshape(-1))


def _weights(cs):
    """(array kept alive by the caller, pointer or None): the weights of a
    rational curve or surface set (attribute ``weights``, one per control
    point), or None for a non-rational one."""
    w = getattr(cs, "weights", None)
    if w is None:
        return None, None
    w = _a(w, np.float64)
    assert w.shape == (len(cs.cps),), w.shape
    return w, w.ctypes.data


def _surf_args(ss):
    return (int(len(ss.deg_u)), _a(ss.deg_u, np.int32), _a(ss.deg_v, np.int32), _a(ss.n_u, np.int32),
            _a(ss.n_v, np.int32), _a(ss.knot_u_off, np.int64), _a(ss.knots_u, np.float64),
            _a(ss.knot_v_off, np.int64), _a(ss.knots_v, np.float64), _a(ss.cp_off, np.int64),
            _a(ss.cps, np.float64).reshape(-1))


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- evaluation

def basis(p, U, t):
    """(span, N_{span-p..span,p}(t)) by the Cox-de Boor recursion (Eq. bsplinebasis)."""
    U = _a(U, np.float64)
    N = np.zeros(p + 1)
    s = C.c_int()
    rc = lib().orc_basis(p, U, len(U), float(t), C.byref(s), N)
    assert rc == OK
    return s.value, N


def eval_curves(cs, qc, t):
    """C, C', C'' at t for curves qc: arrays [nq][3] each."""
    qc = _a(qc, np.int32)
    t = _a(t, np.float64)
    out = np.zeros((len(qc), 3, 3))
    w, wp = _weights(cs)
    rc = lib().orc_eval_curves(*_curve_args(cs), wp, len(qc), qc, t, out.reshape(-1))
    assert rc == OK, rc
    return out[:, 0], out[:, 1], out[:, 2]


def eval_surfaces(ss, qs, uv):
    """S, Su, Sv, Suu, Suv, Svv at (u,v): arrays [nq][3] each."""
    qs = _a(qs, np.int32)
    uv = _a(uv, np.float64).reshape(-1, 2)
    out = np.zeros((len(qs), 6, 3))
    w, wp = _weights(ss)
    rc = lib().orc_eval_surfaces(*_surf_args(ss), wp, len(qs), qs, uv.reshape(-1), out.reshape(-1))
    assert rc == OK, rc
    return tuple(out[:, k] for k in range(6))


# ------------------------------------------------------------- decomposition

def boehm_bezier(p, U, P):
    """Bezier points of every non-empty span by textbook knot insertion: [ns][p+1][3]."""
    U = _a(U, np.float64)
    P = _a(P, np.float64).reshape(-1)
    cap = len(U)
    Q = np.zeros(cap * (p + 1) * 3)
    ns = C.c_int64()
    rc = lib().orc_boehm_bezier(p, U, len(U), P, len(P) // 3, Q, cap, C.byref(ns))
    assert rc == OK, rc
    return Q[: ns.value * (p + 1) * 3].reshape(ns.value, p + 1, 3)


def span_bezier(p, U, P):
    """Bezier points of every non-empty span by the paper's matrix route: [ns][p+1][3]."""
    U = _a(U, np.float64)
    P = _a(P, np.float64).reshape(-1)
    cap = len(U)
    Q = np.zeros(cap * (p + 1) * 3)
    ns = C.c_int64()
    rc = lib().orc_span_bezier(p, U, len(U), P, len(P) // 3, Q, cap, C.byref(ns))
    assert rc == OK, rc
    return Q[: ns.value * (p + 1) * 3].reshape(ns.value, p + 1, 3)


def span_blossom(p, U, P):
    """Bezier points of every non-empty span from the blossom (de Boor's
    algorithm at the span's end knots): [ns][p+1][3]."""
    U = _a(U, np.float64)
    P = _a(P, np.float64).reshape(-1)
    cap = len(U)
    Q = np.zeros(cap * (p + 1) * 3)
    ns = C.c_int64()
    rc = lib().orc_span_blossom(p, U, len(U), P, len(P) // 3, Q, cap, C.byref(ns))
    assert rc == OK, rc
    return Q[: ns.value * (p + 1) * 3].reshape(ns.value, p + 1, 3)


def reduce_g1(Q, variant=0):
    """(R [4][3], delta0, delta1, regular) for a degree-p > 3 Bezier Q [p+1][3]."""
    Q = _a(Q, np.float64)
    p = Q.shape[0] - 1
    R = np.zeros(12)
    d = np.zeros(3)
    rc = lib().orc_reduce_g1(p, Q.reshape(-1), R, d, variant)
    assert rc == OK, rc
    return R.reshape(4, 3), d[0], d[1], bool(d[2])


def to_cubic(Q):
    Q = _a(Q, np.float64)
    R = np.zeros(12)
    rc = lib().orc_to_cubic(Q.shape[0] - 1, Q.reshape(-1), R)
    assert rc == OK
    return R.reshape(4, 3)


def bound2(Q, R):
    Q = _a(Q, np.float64)
    return float(lib().orc_bound2(Q.shape[0] - 1, Q.reshape(-1), _a(R, np.float64).reshape(-1)))


def halve(Q):
    Q = _a(Q, np.float64)
    p = Q.shape[0] - 1
    L = np.zeros((p + 1) * 3)
    R = np.zeros((p + 1) * 3)
    rc = lib().orc_halve(p, Q.reshape(-1), L, R)
    assert rc == OK
    return L.reshape(p + 1, 3), R.reshape(p + 1, 3)


def elevate(Q):
    Q = _a(Q, np.float64)
    n = Q.shape[0] - 1
    E = np.zeros((n + 2) * 3)
    rc = lib().orc_elevate(n, Q.reshape(-1), E)
    assert rc == OK
    return E.reshape(n + 2, 3)


def rspan_bezier(p, U, P, w):
    """Homogeneous Bezier points (W_j Q_j, W_j) of every non-empty span of a
    rational curve by the matrix route: [ns][p+1][4]."""
    U = _a(U, np.float64)
    P = _a(P, np.float64).reshape(-1)
    w = _a(w, np.float64)
    cap = len(U)
    H = np.zeros(cap * (p + 1) * 4)
    ns = C.c_int64()
    rc = lib().orc_rspan_bezier(p, U, len(U), P, w, len(w), H, cap, C.byref(ns))
    assert rc == OK, rc
    return H[: ns.value * (p + 1) * 4].reshape(ns.value, p + 1, 4)


def rhermite(H):
    """C1 Hermite cubic [4][3] of the rational piece H [p+1][4]."""
    H = _a(H, np.float64)
    R = np.zeros(12)
    rc = lib().orc_rhermite(H.shape[0] - 1, H.reshape(-1), R)
    assert rc == OK
    return R.reshape(4, 3)


def rbound2(H, R):
    """Certified bound of max_u |C(u) - R(u)|^2 for the rational piece H and the cubic R."""
    H = _a(H, np.float64)
    return float(lib().orc_rbound2(H.shape[0] - 1, H.reshape(-1), _a(R, np.float64).reshape(-1)))


def rhalve(H):
    H = _a(H, np.float64)
    p = H.shape[0] - 1
    L = np.zeros((p + 1) * 4)
    R = np.zeros((p + 1) * 4)
    rc = lib().orc_rhalve(p, H.reshape(-1), L, R)
    assert rc == OK
    return L.reshape(p + 1, 4), R.reshape(p + 1, 4)


def curve_deriv_bounds(p, U, P, w, q):
    """(V, A): the oracle's bounds of |C'| and |C''| on span q (w None: non-rational)."""
    U = _a(U, np.float64)
    P = _a(P, np.float64).reshape(-1)
    wa = None if w is None else _a(w, np.float64)
    V, A = C.c_double(), C.c_double()
    rc = lib().orc_curve_deriv_bounds(p, U, len(U), P, None if wa is None else wa.ctypes.data, int(q), C.byref(V),
                                      C.byref(A))
    assert rc == OK, rc
    return V.value, A.value


def rsurf_hermite(H):
    """Bicubic Hermite patch [4][4][3] of the rational piece H [pu+1][pv+1][4]."""
    H = _a(H, np.float64)
    R = np.zeros(48)
    rc = lib().orc_rsurf_hermite(H.shape[0] - 1, H.shape[1] - 1, H.reshape(-1), R)
    assert rc == OK
    return R.reshape(4, 4, 3)


def rsurf_bound2(H, R):
    """Certified bound of max |S - R|^2 for the rational piece H and the bicubic R."""
    H = _a(H, np.float64)
    return float(lib().orc_rsurf_bound2(H.shape[0] - 1, H.shape[1] - 1, H.reshape(-1),
                                        _a(R, np.float64).reshape(-1)))


class Decomposition:
    """seg_off [n+1], ctrl [nseg][4][3] (surfaces [nseg][4][4][3]), prange [nseg][2] ([nseg][4])."""

    def __init__(self, seg_off, ctrl, prange, maxdepth, status):
        self.seg_off, self.ctrl, self.prange, self.maxdepth, self.status = seg_off, ctrl, prange, maxdepth, status

    @property
    def total(self):
        return int(self.seg_off[-1])


def decompose_curves(cs, tol_rel, count_only=False):
    args = _curve_args(cs)
    n = args[0]
    seg_off = np.zeros(n + 1, dtype=np.int64)
    tot = C.c_int64()
    md = C.c_int()
    w, wp = _weights(cs)
    rc = lib().orc_decompose_curves(*args, wp, float(tol_rel), seg_off, 0, None, None, C.byref(tot), C.byref(md))
    if rc == EINVAL:
        raise ValueError("invalid curve set")
    if count_only:
        return Decomposition(seg_off, None, None, md.value, rc)
    cap = max(tot.value, 1)
    ctrl = np.zeros(cap * 12)
    prange = np.zeros(cap * 2)
    rc = lib().orc_decompose_curves(*args, wp, float(tol_rel), seg_off, cap, ctrl.ctypes.data, prange.ctypes.data,
                                    C.byref(tot), C.byref(md))
    assert rc in (OK, ENOTCONV), rc
    n_s = tot.value
    return Decomposition(seg_off, ctrl[: n_s * 12].reshape(n_s, 4, 3), prange[: n_s * 2].reshape(n_s, 2),
                         md.value, rc)


def decompose_surfaces(ss, tol_rel, count_only=False):
    args = _surf_args(ss)
    n = args[0]
    seg_off = np.zeros(n + 1, dtype=np.int64)
    tot = C.c_int64()
    md = C.c_int()
    w, wp = _weights(ss)
    rc = lib().orc_decompose_surfaces(*args, wp, float(tol_rel), seg_off, 0, None, None, C.byref(tot),
                                      C.byref(md))
    if rc == EINVAL:
        raise ValueError("invalid surface set")
    if count_only:
        return Decomposition(seg_off, None, None, md.value, rc)
    cap = max(tot.value, 1)
    ctrl = np.zeros(cap * 48)
    prange = np.zeros(cap * 4)
    rc = lib().orc_decompose_surfaces(*args, wp, float(tol_rel), seg_off, cap, ctrl.ctypes.data,
                                      prange.ctypes.data, C.byref(tot), C.byref(md))
    assert rc in (OK, ENOTCONV), rc
    n_s = tot.value
    return Decomposition(seg_off, ctrl[: n_s * 48].reshape(n_s, 4, 4, 3), prange[: n_s * 4].reshape(n_s, 4),
                         md.value, rc)


# ---------------------------------------------------------------- projection

def project_curves(cs, qc, q, nthreads=0):
    """(t*, d*) minimising |q - C(t)| on the original curves (Eq. projections)."""
    qc = _a(qc, np.int32)
    q = _a(q, np.float64).reshape(-1, 3)
    t = np.zeros(len(qc))
    d = np.zeros(len(qc))
    w, wp = _weights(cs)
    rc = lib().orc_project_curves(*_curve_args(cs), wp, len(qc), qc, q.reshape(-1), t, d, int(nthreads))
    assert rc == OK, rc
    return t, d


def project_surfaces(ss, qs, q, nthreads=0):
    """((u*,v*), d*) minimising |q - S(u,v)| on the original surfaces."""
    qs = _a(qs, np.int32)
    q = _a(q, np.float64).reshape(-1, 3)
    uv = np.zeros((len(qs), 2))
    d = np.zeros(len(qs))
    w, wp = _weights(ss)
    rc = lib().orc_project_surfaces(*_surf_args(ss), wp, len(qs), qs, q.reshape(-1), uv.reshape(-1), d,
                                    int(nthreads))
    assert rc == OK, rc
    return uv, d


def surf_deriv_bounds(pu, pv, U, V, P, w, qu, qv):
    """(Vu, Vv, Auu, Avv): the oracle's bounds of |S_u|, |S_v|, |S_uu|, |S_vv|
    on span pair (qu, qv); P [nu][nv][3], w [nu][nv] or None."""
    P = _a(P, np.float64)
    nu, nv = P.shape[0], P.shape[1]
    wa = None if w is None else _a(w, np.float64).reshape(-1)
    out = np.zeros(4)
    rc = lib().orc_surf_deriv_bounds(pu, pv, _a(U, np.float64), nu, _a(V, np.float64), nv, P.reshape(-1),
                                     None if wa is None else wa.ctypes.data, int(qu), int(qv), out)
    assert rc == OK, rc
    return tuple(out)


def curve_diag(cs):
    """Per-curve diagonal of the control-point box."""
    lo = np.minimum.reduceat(cs.cps, cs.cp_off[:-1], axis=0)
    hi = np.maximum.reduceat(cs.cps, cs.cp_off[:-1], axis=0)
    return np.linalg.norm(hi - lo, axis=1)


def surface_diag(ss):
    lo = np.minimum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    hi = np.maximum.reduceat(ss.cps, ss.cp_off[:-1], axis=0)
    return np.linalg.norm(hi - lo, axis=1)


# ------------------------------------------------------------------- tables
# The paper's constant matrices, written out from their definitions.

class tables:
    @staticmethod
    def S(z):
        """8x4 cubic subdivision matrix [S_L(z); S_R(z)] as printed in Sec. 4.2.2
        (Eq. subLandR): (S_L)_{ij} = C(i,j) z^j (1-z)^{i-j};
        (S_R)_{ij} = C(3-i, j-i) z^{j-i} (1-z)^{3-j} (printed matrix; the
        index formula printed beside it swaps the exponents)."""
        SL = np.zeros((4, 4))
        SR = np.zeros((4, 4))
        for i in range(4):
            for j in range(i + 1):
                SL[i, j] = math.comb(i, j) * z ** j * (1 - z) ** (i - j)
            for j in range(i, 4):
                SR[i, j] = math.comb(3 - i, j - i) * z ** (j - i) * (1 - z) ** (3 - j)
        return np.vstack([SL, SR])

    @staticmethod
    def T(n):
        """Power -> Bernstein matrix, b = T a (Sec. 4.3): T_ij = C(i,j)/C(n,j), j <= i
        (the printed 6x6 matrix; the index formula printed beside it divides by
        C(n,i) instead)."""
        T = np.zeros((n + 1, n + 1))
        for i in range(n + 1):
            for j in range(i + 1):
                T[i, j] = math.comb(i, j) / math.comb(n, j)
        return T

    @staticmethod
    def bernstein_to_power(n):
        """M with a = M b: M_kj = C(n,j) C(n-j,k-j) (-1)^(k-j) (appendix, power-to-Bernstein section)."""
        M = np.zeros((n + 1, n + 1))
        for k in range(n + 1):
            for j in range(k + 1):
                M[k, j] = math.comb(n, j) * math.comb(n - j, k - j) * (-1) ** (k - j)
        return M

    @staticmethod
    def gram(m, n):
        """G_{m,n}: g_ij = C(m,i) C(n,j) / ((m+n+1) C(m+n,i+j)) (Eq. gram)."""
        G = np.zeros((m + 1, n + 1))
        for i in range(m + 1):
            for j in range(n + 1):
                G[i, j] = math.comb(m, i) * math.comb(n, j) / ((m + n + 1) * math.comb(m + n, i + j))
        return G

    @staticmethod
    def M_qpT(tq, tq1, p):
        """Reparameterisation matrix with T = U M (Eq. Mqpt), entries
        m_ji = C(i,j) (t_{q+1}-t_q)^j t_q^(i-j) for j <= i (Eq. appMelement)."""
        d = tq1 - tq
        M = np.zeros((p + 1, p + 1))
        for i in range(p + 1):
            for j in range(i + 1):
                M[j, i] = math.comb(i, j) * d ** j * tq ** (i - j)
        return M

    @staticmethod
    def A_qpT_exact(U, q, p):
        """A_{q,p,T} in exact rational arithmetic (fractions.Fraction): a list of
        p+1 columns of coefficient lists, same recursion as A_qpT."""
        from fractions import Fraction as F

        def pmul(a, b):
            out = [F(0)] * (len(a) + len(b) - 1)
            for i, x in enumerate(a):
                for j, y in enumerate(b):
                    out[i + j] += x * y
            return out

        def padd(a, b):
            n = max(len(a), len(b))
            return [(a[i] if i < len(a) else F(0)) + (b[i] if i < len(b) else F(0)) for i in range(n)]

        Uf = [F(float(x)) for x in U]
        cur = [[F(1)]]
        for k in range(1, p + 1):
            nxt = []
            for j in range(k + 1):
                i = q - k + j
                acc = [F(0)]
                if j >= 1 and Uf[i + k] != Uf[i]:
                    den = Uf[i + k] - Uf[i]
                    acc = padd(acc, pmul([-Uf[i] / den, 1 / den], cur[j - 1]))
                if j <= k - 1 and Uf[i + k + 1] != Uf[i + 1]:
                    den = Uf[i + k + 1] - Uf[i + 1]
                    acc = padd(acc, pmul([Uf[i + k + 1] / den, -1 / den], cur[j]))
                nxt.append(acc)
            cur = nxt
        A = [[F(0)] * (p + 1) for _ in range(p + 1)]
        for k, c in enumerate(cur):
            for e, x in enumerate(c):
                A[e][k] = x
        return A

    @staticmethod
    def decomfinal_exact(U, q, p, P):
        """Q = B_p^{-1} M_{q,p,T} A_{q,p,T} [P_{q-p}..P_q] evaluated exactly in
        rationals (Eq. decomfinal), returned as float64 [p+1][3]."""
        from fractions import Fraction as F
        A = tables.A_qpT_exact(U, q, p)
        tq, d = F(float(U[q])), F(float(U[q + 1])) - F(float(U[q]))
        M = [[F(math.comb(i, j)) * d ** j * tq ** (i - j) if j <= i else F(0) for i in range(p + 1)]
             for j in range(p + 1)]
        Tm = [[F(math.comb(i, j), math.comb(p, j)) if j <= i else F(0) for j in range(p + 1)] for i in range(p + 1)]
        Pl = [[F(float(x)) for x in P[q - p + r]] for r in range(p + 1)]

        def mm(X, Y):
            return [[sum(X[i][k] * Y[k][j] for k in range(len(Y))) for j in range(len(Y[0]))] for i in range(len(X))]

        Q = mm(Tm, mm(M, mm(A, Pl)))
        return np.array([[float(x) for x in row] for row in Q])

    @staticmethod
    def A_qpT(U, q, p):
        """Global power-basis coefficient matrix A_{q,p,T} of Eq. bsplinematrix:
        C(t) = [1 t ... t^p] A [P_{q-p} .. P_q]^T on [t_q, t_{q+1}].  Column k
        holds the coefficients of N_{q-p+k,p}(t), built by the Cox-de Boor
        recursion (Eq. bsplinebasis) on polynomials in t."""
        from numpy.polynomial import polynomial as Pn
        cur = [np.array([1.0])]  # N_{q,0}
        for k in range(1, p + 1):
            nxt = []
            for j in range(k + 1):
                i = q - k + j
                acc = np.zeros(1)
                if j >= 1 and U[i + k] != U[i]:
                    acc = Pn.polyadd(acc, Pn.polymul(np.array([-U[i], 1.0]) / (U[i + k] - U[i]), cur[j - 1]))
                if j <= k - 1 and U[i + k + 1] != U[i + 1]:
                    acc = Pn.polyadd(acc, Pn.polymul(np.array([U[i + k + 1], -1.0]) / (U[i + k + 1] - U[i + 1]),
                                                     cur[j]))
                nxt.append(acc)
            cur = nxt
        A = np.zeros((p + 1, p + 1))
        for k, c in enumerate(cur):
            A[: len(c), k] = c
        return A
