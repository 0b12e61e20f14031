"""FP64 reference of the warm-start network.  TEST INFRASTRUCTURE.

The network, loss and features follow the definitions stated in include/drot.h
(drot_mlp_*), written here plainly in NumPy, in FP64, with no BF16 rounding:
only the tests use this module, to check the GPU forward pass, the gradients
of the training step and the feature rows.
"""

from __future__ import annotations

import numpy as np

IN = 64
WIDTH = 256
SHAPES = [("W1", (WIDTH, IN)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (WIDTH,)), ("b4", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    params = np.asarray(params, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = params[off:off + k].reshape(shape)
        off += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(params, F):
    P = unpack(params)
    F = np.asarray(F, dtype=np.float64)
    A1 = F @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    A3 = H2 @ P["W3"].T + P["b3"]
    H3 = np.maximum(A3, 0.0)
    out = H3 @ P["W4"] + P["b4"][0]
    return out, (F, H1, H2, H3)


def loss(out, y, w, seg, nseg):
    """(1/S) sum_s sum_{r in s} w_r (e_r - ebar_s)^2 with e = out - y, ebar_s the w-weighted mean of e over s."""
    out = np.asarray(out, dtype=np.float64)
    e = out - np.asarray(y, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    seg = np.asarray(seg)
    L = 0.0
    g = np.zeros_like(out)
    for s in range(nseg):
        idx = seg == s
        if not idx.any():
            continue
        eb = (w[idx] * e[idx]).sum() / w[idx].sum()
        L += (w[idx] * (e[idx] - eb) ** 2).sum()
        g[idx] = 2.0 * w[idx] * (e[idx] - eb)
    return L / nseg, g / nseg


def loss_and_grad(params, F, y, w, seg, nseg):
    P = unpack(params)
    out, (F, H1, H2, H3) = forward(params, F)
    L, g = loss(out, y, w, seg, nseg)
    grads = {}
    grads["W4"] = H3.T @ g
    grads["b4"] = np.array([g.sum()])
    D3 = np.outer(g, P["W4"]) * (H3 > 0)
    grads["W3"] = D3.T @ H2
    grads["b3"] = D3.sum(0)
    D2 = (D3 @ P["W3"]) * (H2 > 0)
    grads["W2"] = D2.T @ H1
    grads["b2"] = D2.sum(0)
    D1 = (D2 @ P["W2"]) * (H1 > 0)
    grads["W1"] = D1.T @ F
    grads["b1"] = D1.sum(0)
    return L, pack(grads)


def features(x, y, p, q):
    """Feature rows of the source points (the layout stated for drot_mlp_features)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = len(x)

    def cell(v):
        return np.clip((v * 4.0).astype(np.int64), 0, 3)

    hs = np.zeros(16)
    np.add.at(hs, 4 * cell(x[:, 0]) + cell(x[:, 1]), p)
    ht = np.zeros(16)
    np.add.at(ht, 4 * cell(y[:, 0]) + cell(y[:, 1]), q)
    ms = (p[:, None] * x).sum(0)
    mt = (q[:, None] * y).sum(0)
    exx = (q * y[:, 0] ** 2).sum() - mt[0] ** 2
    eyy = (q * y[:, 1] ** 2).sum() - mt[1] ** 2
    exy = (q * y[:, 0] * y[:, 1]).sum() - mt[0] * mt[1]
    F = np.zeros((m, IN))
    F[:, 0:2] = x
    F[:, 2] = m * p
    F[:, 3:19] = hs
    F[:, 19:35] = ht
    F[:, 35:37] = ms
    F[:, 37:39] = mt
    F[:, 39] = exx
    F[:, 40] = eyy
    F[:, 41] = exy
    F[:, 42] = 1.0
    return F
