"""FP64 oracle of the learned far-field correction -- TEST INFRASTRUCTURE.

Only tests/ and bench.py's reference arm use it; the product library never
does.  Plain numpy, written from the definitions:

* features(tf, pos, eps): the 12 rotation-invariant inputs of every body
  from an oracle tree evaluation -- log|a|, log(-phi), log(1 + accepted
  cells) in the level bins 0-3, 4-6, 7-9, 10-21, log(1 + body-body
  interactions), log(n_G / (e_G^3 + eps^3)), log((d_G + eps)/eps) with e_G the
  largest extent and d_G the diagonal of the group's bounding box, |o| /
  (d_G / 2) and the cosine between o and a, o the body's offset from the box
  centre, log n_G;
* frame(...): the body-local frame e0 = a/|a|, e1 = unit part of o
  orthogonal to e0 (the least-aligned coordinate axis if o is zero or along
  e0), e2 = e0 x e1; the network's 3 outputs are coefficients of the
  residual (a_direct - a)/|a| along it (labels());
* forward(P, norm, X): the network 12 -> 64 -> 64 -> 3 with ReLU, inputs
  (x - mu)/sigma, then inputs, weight matrices and hidden activations rounded
  to bfloat16 (round to nearest even from float32), FP64 sums;
* loss_grad(P, norm, X, Y): loss mean((net - Y/ysig)^2) over rows and the 3
  outputs and its analytic gradient (rounding passed straight through).
Parameters P (5187): W1 64x12, b1 64, W2 64x64, b2 64, W3 3x64, b3 3
(rows W[out][in]); norm (25): mu[12], sigma[12], ysig.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 12, 64, 3
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) via float32, back to float64."""
    b = np.asarray(x, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(P) -> dict:
    P = np.asarray(P, np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = P[o:o + k].reshape(shp)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def forward(P, norm, X, rounded: bool = True):
    """Returns (y, cache) for rows X (n x 12 raw features)."""
    r = bf16 if rounded else (lambda v: np.asarray(v, np.float64))
    w = unpack(P)
    norm = np.asarray(norm, np.float64)
    xn = (np.asarray(X, np.float64) - norm[:IN]) / norm[IN:2 * IN]
    x = r(xn)
    W1, W2, W3 = r(w["W1"]), r(w["W2"]), r(w["W3"])
    z1 = x @ W1.T + w["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + w["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ W3.T + w["b3"]
    return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, W3=W3)


def loss_grad(P, norm, X, Y, rounded: bool = True):
    norm = np.asarray(norm, np.float64)
    y, c = forward(P, norm, X, rounded)
    t = np.asarray(Y, np.float64) / norm[2 * IN]
    n = y.shape[0]
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / (OUT * n)
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(0)}
    dh2 = (dy @ c["W3"]) * (c["z2"] > 0)
    g["W2"] = dh2.T @ c["h1"]
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ c["W2"]) * (c["z1"] > 0)
    g["W1"] = dh1.T @ c["x"]
    g["b1"] = dh1.sum(0)
    return loss, pack(g)


def _groups(tf, pos):
    pos = np.asarray(pos, np.float32)
    sp = pos[tf.perm]
    lo = np.minimum.reduceat(sp, tf.gbeg, axis=0).astype(np.float64)
    hi = np.maximum.reduceat(sp, tf.gbeg, axis=0).astype(np.float64)
    g = tf.group_of
    off = pos.astype(np.float64) - 0.5 * (lo + hi)[g]
    return lo, hi, g, off


def frame(a, off):
    """Body-local frame (e0, e1, e2), each (n, 3)."""
    a = np.asarray(a, np.float64)
    an = np.linalg.norm(a, axis=1)
    e0 = np.where(an[:, None] > 0, a / np.maximum(an, 1e-300)[:, None], np.array([1.0, 0.0, 0.0]))
    on = np.linalg.norm(off, axis=1)
    p = off - (off * e0).sum(1, keepdims=True) * e0
    pn = np.linalg.norm(p, axis=1)
    bad = ~((pn > 1e-6 * on) & (pn > 0))
    if bad.any():
        ax = np.argmin(np.abs(e0[bad]), axis=1)          # first least-aligned axis
        u = np.eye(3)[ax]
        p[bad] = u - (u * e0[bad]).sum(1, keepdims=True) * e0[bad]
        pn[bad] = np.linalg.norm(p[bad], axis=1)
    e1 = p / pn[:, None]
    return e0, e1, np.cross(e0, e1)


def features(tf, pos, eps: float) -> np.ndarray:
    """12 raw inputs per body (caller order) of an oracle tree evaluation."""
    a = tf.acc
    an = np.linalg.norm(a, axis=1)
    lo, hi, g, off = _groups(tf, pos)
    ext = hi - lo
    emax = ext.max(1)
    diag = np.sqrt((ext ** 2).sum(1))
    e0, _, _ = frame(a, off)
    on = np.linalg.norm(off, axis=1)
    X = np.zeros((a.shape[0], IN))
    X[:, 0] = np.log(np.maximum(an, 1e-30))
    X[:, 1] = np.log(np.maximum(-tf.pot, 1e-30))
    X[:, 2:6] = np.log1p(tf.npc_bins)
    X[:, 6] = np.log1p(tf.n_pp)
    X[:, 7] = np.log(tf.gcnt[g] / (emax[g] ** 3 + eps ** 3))
    X[:, 8] = np.log((diag[g] + eps) / eps)
    X[:, 9] = np.where(diag[g] > 0, on / np.maximum(0.5 * diag[g], 1e-300), 0.0)
    X[:, 10] = np.where(on > 0, (off * e0).sum(1) / np.maximum(on, 1e-300), 0.0)
    X[:, 11] = np.log(tf.gcnt[g])
    return X


def labels(tf, pos, a_direct, idx) -> np.ndarray:
    """Targets at bodies idx: (r.e0, r.e1, r.e2), r = (a_direct - a)/|a|."""
    a = tf.acc[idx]
    _, _, _, off = _groups(tf, pos)
    e0, e1, e2 = frame(a, off[idx])
    r = (np.asarray(a_direct, np.float64) - a) / np.linalg.norm(a, axis=1)[:, None]
    return np.stack([(r * e0).sum(1), (r * e1).sum(1), (r * e2).sum(1)], 1)
