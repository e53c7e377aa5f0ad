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

_K = math.sqrt(2.0 / math.pi)
_C = 0.044715


def unpack(theta):
    """Parameter vector -> dict of arrays (views)."""
    out, o = {}, 0
    for name, shp in _SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p, total=NPARAM):
    theta = np.zeros(total)
    o = 0
    for name, shp in _SHAPES:
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
    """p: dict of layer arrays (any widths), X [n][in].  Returns t [n] and
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
    z4 = r(Hs[-1]) @ r(p["w4"]) + p["b4"][0]
    return sigmoid(z4), Zs, Hs


def loss_and_grads(p, X, y):
    """Mean squared error of t against y and its gradient, by the chain rule
    written out layer by layer."""
    t, Zs, Hs = forward(p, X)
    n = len(y)
    r = t - y
    loss = float(np.mean(r * r))
    dz4 = (2.0 / n) * r * t * (1.0 - t)
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
