"""FP64 reference of the learned Newton seed -- TEST INFRASTRUCTURE ONLY.

Plain NumPy, no blocking or fusion: the small MLP that maps a (segment,
query) pair to a starting parameter, its loss and gradients, the Adam update,
the pair features, and the label the network is trained on (the minimiser of
the squared distance on one cubic Bezier segment).

The paper has no learned component; the network stands in for the coarse
search stage that seeds Newton's method on D(t) = |C(t) - q|^2 (Sec. 3,
Eqs. Dt, Et, E't).  Definitions used here:

* network 15 -> 128 -> 128 -> 128 -> 1 (input padded with one zero to 16),
  GELU in its tanh form g(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))
  after each hidden layer, logistic sigmoid on the output, so t in (0, 1);
* loss: mean over the batch of (t - t*)^2;
* Adam (Kingma & Ba) with bias correction, applied to every parameter;
* features of a cubic Bezier segment P0..P3 and query q, in the frame of the
  segment's control-point box (centre c, scale s = 1 / longest side, no
  rotation): (P_i - c) s for i = 0..3, then the query v = (q - c) s with
  its part across the chord P0 -> P3 shortened to length min(1, |part|)
  (the part along the chord, which fixes the minimiser of a far query, is
  kept), then a zero;
* label: the global minimiser of |C(u) - q|^2 on u in [0, 1] (ties -> the
  smaller u).

Parameter vector layout (FP32 on the device, FP64 here): W1 [128][16], b1,
W2 [128][128], b2, W3 [128][128], b3, w4 [128], b4, then 3 zeros.
"""
from __future__ import annotations

import math

import numpy as np

H = 128
IN = 16
NPARAM = 35332
_SHAPES = (("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
           ("w4", (H,)), ("b4", (1,)))
# the surface network: 64 inputs (51 used) -> 2 outputs (u, v)
SIN = 64
SNPARAM = 41604
SHAPES_SURF = (("W1", (H, SIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
               ("W4", (2, H)), ("b4", (2,)))

_K = math.sqrt(2.0 / math.pi)
_C = 0.044715


def unpack(theta, shapes=_SHAPES):
    """Parameter vector -> dict of arrays (views)."""
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p, total=NPARAM, shapes=_SHAPES):
    theta = np.zeros(total)
    o = 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        theta[o:o + n] = np.asarray(p[name], np.float64).reshape(-1)
        o += n
    return theta


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_K * (x + _C * x ** 3)))


def gelu_grad(x):
    th = np.tanh(_K * (x + _C * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * _K * (1.0 + 3.0 * _C * x * x)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, bf16=False):
    """p: dict of layer arrays (any widths), X [n][in].  Returns t [n] (one
    output: w4 [H], b4 [1]) or t [n][k] (k outputs: W4 [k][H], b4 [k]) and
    the pre-activations (Z1, Z2, Z3) and activations (H0 = X, H1, H2, H3).
    bf16=True evaluates the network at the precision it is served in: every
    weight matrix and every layer input rounded to bfloat16 (biases and the
    accumulation stay in full precision)."""
    r = round_bf16 if bf16 else (lambda a: a)
    Hs, Zs = [np.asarray(X, np.float64)], []
    for W, b in ((p["W1"], p["b1"]), (p["W2"], p["b2"]), (p["W3"], p["b3"])):
        Z = r(Hs[-1]) @ r(W).T + b
        Zs.append(Z)
        Hs.append(gelu(Z))
    if "W4" in p:
        return sigmoid(r(Hs[-1]) @ r(p["W4"]).T + p["b4"]), Zs, Hs
    z4 = r(Hs[-1]) @ r(p["w4"]) + p["b4"][0]
    return sigmoid(z4), Zs, Hs


def loss_and_grads(p, X, y):
    """Mean squared error of t against y (the mean over rows and outputs)
    and its gradient, by the chain rule written out layer by layer."""
    t, Zs, Hs = forward(p, X)
    r = t - y
    loss = float(np.mean(r * r))
    dz4 = (2.0 / r.size) * r * t * (1.0 - t)
    if "W4" in p:
        g = {"W4": dz4.T @ Hs[3], "b4": dz4.sum(axis=0)}
        dH = dz4 @ p["W4"]
    else:
        g = {"w4": Hs[3].T @ dz4, "b4": np.array([dz4.sum()])}
        dH = np.outer(dz4, p["w4"])
    for li in (3, 2, 1):
        dZ = dH * gelu_grad(Zs[li - 1])
        g[f"W{li}"] = dZ.T @ Hs[li - 1]
        g[f"b{li}"] = dZ.sum(axis=0)
        dH = dZ @ p[f"W{li}"]
    return loss, g


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(ctrl, q):
    """ctrl [n][4][3] Bezier control points, q [n][3] -> X [n][16]."""
    ctrl = np.asarray(ctrl, np.float64)
    q = np.asarray(q, np.float64)
    lo, hi = ctrl.min(axis=1), ctrl.max(axis=1)
    c = 0.5 * (lo + hi)
    ext = (hi - lo).max(axis=1)
    s = np.where(ext > 0, 1.0 / np.where(ext > 0, ext, 1.0), 1.0)
    X = np.zeros((len(q), IN))
    X[:, :12] = ((ctrl - c[:, None, :]) * s[:, None, None]).reshape(-1, 12)
    v = (q - c) * s[:, None]
    # query: its coordinate along the chord P0 -> P3 kept, the part across
    # the chord shortened to length <= 1
    ch = ctrl[:, 3] - ctrl[:, 0]
    ln = np.linalg.norm(ch, axis=1)
    d = np.where(ln[:, None] > 0, ch / np.where(ln > 0, ln, 1.0)[:, None], np.array([1.0, 0.0, 0.0]))
    a = np.einsum("ij,ij->i", v, d)
    w = v - a[:, None] * d
    r = np.linalg.norm(w, axis=1)
    X[:, 12:15] = a[:, None] * d + w / np.maximum(1.0, r)[:, None]
    return X


def _bezier(P, u):
    u = np.asarray(u)[..., None]
    w = 1.0 - u
    return w ** 3 * P[0] + 3 * w * w * u * P[1] + 3 * w * u * u * P[2] + u ** 3 * P[3]


def _bezier_d(P, u):
    u = np.asarray(u)[..., None]
    w = 1.0 - u
    return 3 * (w * w * (P[1] - P[0]) + 2 * w * u * (P[2] - P[1]) + u * u * (P[3] - P[2]))


def _bezier_dd(P, u):
    u = np.asarray(u)[..., None]
    return 6 * ((1.0 - u) * (P[2] - 2 * P[1] + P[0]) + u * (P[3] - 2 * P[2] + P[1]))


def segment_minimiser(P, q, samples=513):
    """Global minimiser of |C(u) - q|^2 on [0, 1] for one cubic Bezier
    segment: dense sampling, safeguarded Newton on E = (C - q).C' from every
    sampled local minimum, both ends as candidates; ties -> smaller u."""
    P = np.asarray(P, np.float64)
    q = np.asarray(q, np.float64)
    us = np.linspace(0.0, 1.0, samples)
    D = ((_bezier(P, us) - q) ** 2).sum(axis=1)
    cands = [0.0, 1.0]
    for i in range(1, samples - 1):
        if D[i] <= D[i - 1] and D[i] <= D[i + 1]:
            lo, hi, u = us[i - 1], us[i + 1], us[i]
            for _ in range(100):
                C = _bezier(P, u) - q
                d1 = _bezier_d(P, u)
                E = float(C @ d1)
                Ep = float(d1 @ d1 + C @ _bezier_dd(P, u))
                if E > 0:
                    hi = u
                elif E < 0:
                    lo = u
                else:
                    break
                un = u - E / Ep if Ep > 0 else 0.5 * (lo + hi)
                if not (lo < un < hi):
                    un = 0.5 * (lo + hi)
                if abs(un - u) <= 1e-16 or hi - lo <= 1e-16:
                    u = un
                    break
                u = un
            cands.append(u)
    cands = np.array(sorted(cands))
    Dc = ((_bezier(P, cands) - q) ** 2).sum(axis=1)
    k = int(np.argmin(Dc))
    return float(cands[k]), float(Dc[k])


# ------------------------------------------------------- surface network

def surface_features(ctrl, q):
    """ctrl [n][4][4][3] bicubic Bezier nets (first index along u), q [n][3]
    -> X [n][64]: the 16 control points relative to the centre of their box,
    scaled by 1 / its longest side (i along u, then j, then xyz); the query
    in the same frame with its component along the normal of the frame
    e1 = P30 - P00, e2 = (P03 - P00) without its e1 part clamped to [-1, 1]
    (the tangential components kept); then 13 zeros."""
    ctrl = np.asarray(ctrl, np.float64)
    q = np.asarray(q, np.float64)
    n = len(q)
    d = ctrl - ctrl[:, :1, :1, :]
    lo = np.minimum(d.reshape(n, 16, 3).min(axis=1), 0.0)
    hi = np.maximum(d.reshape(n, 16, 3).max(axis=1), 0.0)
    c = 0.5 * (lo + hi)
    ext = (hi - lo).max(axis=1)
    s = np.where(ext > 0, 1.0 / np.where(ext > 0, ext, 1.0), 1.0)
    X = np.zeros((n, SIN))
    X[:, :48] = ((d - c[:, None, None, :]) * s[:, None, None, None]).reshape(n, 48)
    v = (q - ctrl[:, 0, 0] - c) * s[:, None]
    e1 = d[:, 3, 0]
    l1 = np.linalg.norm(e1, axis=1)
    e1 = np.where(l1[:, None] > 0, e1 / np.where(l1 > 0, l1, 1.0)[:, None], np.array([1.0, 0.0, 0.0]))
    w = d[:, 0, 3] - np.einsum("ij,ij->i", d[:, 0, 3], e1)[:, None] * e1
    l2 = np.linalg.norm(w, axis=1)
    # a degenerate second side: any unit vector across e1
    t = np.where((np.abs(e1[:, 0]) < 0.9)[:, None], np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))
    alt = t - np.einsum("ij,ij->i", t, e1)[:, None] * e1
    alt /= np.linalg.norm(alt, axis=1)[:, None]
    e2 = np.where(l2[:, None] > 0, w / np.where(l2 > 0, l2, 1.0)[:, None], alt)
    nn = np.cross(e1, e2)
    a1 = np.einsum("ij,ij->i", v, e1)
    a2 = np.einsum("ij,ij->i", v, e2)
    a3 = np.clip(np.einsum("ij,ij->i", v, nn), -1.0, 1.0)
    X[:, 48:51] = a1[:, None] * e1 + a2[:, None] * e2 + a3[:, None] * nn
    return X


def _bern3(t):
    t = np.asarray(t, np.float64)
    w = 1.0 - t
    return np.stack([w ** 3, 3 * w * w * t, 3 * w * t * t, t ** 3], axis=-1)


def _bern3_d(t):
    t = np.asarray(t, np.float64)
    w = 1.0 - t
    return np.stack([-3 * w * w, 3 * w * w - 6 * w * t, 6 * w * t - 3 * t * t, 3 * t * t], axis=-1)


def _bern3_dd(t):
    t = np.asarray(t, np.float64)
    return np.stack([6 * (1 - t), -12 + 18 * t, 6 - 18 * t, 6 * t], axis=-1)


def _patch(P, u, v, du=0, dv=0):
    fu = (_bern3, _bern3_d, _bern3_dd)[du](u)
    fv = (_bern3, _bern3_d, _bern3_dd)[dv](v)
    return np.einsum("...i,...j,ijc->...c", fu, fv, P)


def patch_minimiser(P, q, samples=33):
    """Global minimiser of |S(u,v) - q|^2 over (u,v) in [0,1]^2 for one
    bicubic Bezier patch P [4][4][3]: the four corners, the minimiser of each
    edge (a cubic curve: segment_minimiser), and a damped Newton iteration on
    grad D kept inside the square from every local minimum of a dense sample
    grid; the smallest distance wins (ties -> smaller u, then smaller v)."""
    P = np.asarray(P, np.float64)
    q = np.asarray(q, np.float64)
    cands = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (1.0, 1.0)]
    for fixed_u, val in ((True, 0.0), (True, 1.0), (False, 0.0), (False, 1.0)):
        edge = P[0 if val == 0.0 else 3] if fixed_u else P[:, 0 if val == 0.0 else 3]
        t, _ = segment_minimiser(edge, q)
        cands.append((val, t) if fixed_u else (t, val))
    g = np.linspace(0.0, 1.0, samples)
    uu, vv = np.meshgrid(g, g, indexing="ij")
    D = ((_patch(P, uu, vv) - q) ** 2).sum(axis=-1)
    for i in range(samples):
        for j in range(samples):
            nb = D[max(i - 1, 0):i + 2, max(j - 1, 0):j + 2]
            if D[i, j] > nb.min():
                continue
            u, v = g[i], g[j]
            for _ in range(100):
                S = _patch(P, u, v) - q
                Su, Sv = _patch(P, u, v, 1, 0), _patch(P, u, v, 0, 1)
                gr = np.array([S @ Su, S @ Sv])
                Hm = np.array([[Su @ Su + S @ _patch(P, u, v, 2, 0), Su @ Sv + S @ _patch(P, u, v, 1, 1)],
                               [0.0, Sv @ Sv + S @ _patch(P, u, v, 0, 2)]])
                Hm[1, 0] = Hm[0, 1]
                if np.all(np.linalg.eigvalsh(Hm) > 0):
                    step = -np.linalg.solve(Hm, gr)
                else:
                    step = -gr / max(np.linalg.norm(gr), 1e-300) / samples
                D0 = float(S @ S)
                lam, acc = 1.0, False
                for _ in range(60):
                    un, vn = min(max(u + lam * step[0], 0.0), 1.0), min(max(v + lam * step[1], 0.0), 1.0)
                    Sn = _patch(P, un, vn) - q
                    if float(Sn @ Sn) <= D0:
                        acc = True
                        break
                    lam *= 0.5
                if not acc:
                    break
                moved = abs(un - u) + abs(vn - v)
                u, v = un, vn
                if moved <= 1e-16:
                    break
            cands.append((u, v))
    best = None
    for u, v in cands:
        S = _patch(P, u, v) - q
        Dc = float(S @ S)
        key = (Dc, u, v)
        if best is None or key < best:
            best = key
    return best[1], best[2], best[0]
