"""FP64 NumPy statement of the tail network: forward pass, L1 loss and its
gradient by explicit backpropagation.

TEST INFRASTRUCTURE ONLY: the GPU tests compare the library's FP16 training
and inference kernels against these functions. Shares no code with the CUDA
library. The network is the library's own learned tail estimator (the paper
has no network): the definition followed here is the one documented with
the tail-network functions of the C interface (layer shapes, parameter
order, per-beam scale s = max(prior mass, 0.1 x tail bound)).

Shapes: x [B, 5440, 2] (levels of 64^2, 32^2, 16^2, 8^2 cells, row-major,
channels last), rows / target [B, n_coarse + 4].
"""
from __future__ import annotations

import numpy as np

C = 32
HID = 256
K1, K2 = 32, 320
LEVELS = ((0, 64), (4096, 32), (5120, 16), (5376, 8))  # (first cell, side)


def _pad8(n):
    return (n + 7) // 8 * 8


def layout(nc):
    """Offsets and shapes of the parameter tensors in the flat vector."""
    F = 64 * C + 128 + nc
    shapes = [("w1", (C, K1)), ("b1", (C,)), ("w2", (C, K2)), ("b2", (C,)), ("w3", (C, K2)), ("b3", (C,)),
              ("f1", (HID, F)), ("fb1", (HID,)), ("f2", (nc, HID)), ("fb2", (nc,))]
    out, o = {}, 0
    for name, shp in shapes:
        out[name] = (o, shp)
        o += _pad8(int(np.prod(shp)))
    return out, o


def unpack(params, nc):
    lay, n = layout(nc)
    assert params.size == n
    return {k: params[o:o + int(np.prod(s))].reshape(s).astype(np.float64) for k, (o, s) in lay.items()}


def pack(tensors, nc):
    lay, n = layout(nc)
    p = np.zeros(n)
    for k, (o, s) in lay.items():
        p[o:o + int(np.prod(s))] = np.asarray(tensors[k], np.float64).ravel()
    return p


def level(x, i):
    first, side = LEVELS[i]
    return x[:, first:first + side * side, :].reshape(x.shape[0], side, side, 2).astype(np.float64)


def im2col(a):
    """[B, H, W, Cin] -> [B, H/2, W/2, 9 Cin]: 3x3 windows of stride 2 with
    one pixel of zero padding, column tap * Cin + c, tap = 3 ky + kx."""
    B, H, W, Ci = a.shape
    ap = np.zeros((B, H + 2, W + 2, Ci))
    ap[:, 1:-1, 1:-1] = a
    cols = []
    for ky in range(3):
        for kx in range(3):
            cols.append(ap[:, ky:ky + H:2, kx:kx + W:2, :])
    return np.concatenate(cols, axis=3)


def col2im(d, H, W, Ci):
    """Adjoint of im2col."""
    B = d.shape[0]
    ap = np.zeros((B, H + 2, W + 2, Ci))
    for ky in range(3):
        for kx in range(3):
            t = 3 * ky + kx
            ap[:, ky:ky + H:2, kx:kx + W:2, :] += d[..., t * Ci:(t + 1) * Ci]
    return ap[:, 1:-1, 1:-1]


def scale(rows, nc):
    m, e = rows[:, nc + 3], rows[:, nc + 1]
    return np.maximum(m, 0.1 * e)


def forward(params, x, rows, nc):
    P = unpack(params, nc)
    rows = np.asarray(rows, np.float64)
    B = x.shape[0]
    L = [level(x, i) for i in range(4)]
    cache = {"L": L}
    X1 = im2col(L[0])                                  # [B, 32, 32, 18]
    Z1 = X1 @ P["w1"][:, :18].T + P["b1"]
    A1 = np.maximum(Z1, 0)
    X2 = im2col(np.concatenate([A1, L[1]], axis=3))    # [B, 16, 16, 306]
    Z2 = X2 @ P["w2"][:, :306].T + P["b2"]
    A2 = np.maximum(Z2, 0)
    X3 = im2col(np.concatenate([A2, L[2]], axis=3))    # [B, 8, 8, 306]
    Z3 = X3 @ P["w3"][:, :306].T + P["b3"]
    A3 = np.maximum(Z3, 0)
    s = scale(rows, nc)
    pn = np.where(s[:, None] > 0, rows[:, :nc] / np.where(s > 0, s, 1)[:, None], 0.0)
    f = np.concatenate([A3.reshape(B, -1), L[3].reshape(B, -1), pn], axis=1)
    Zh = f @ P["f1"].T + P["fb1"]
    Hh = np.maximum(Zh, 0)
    D = Hh @ P["f2"].T + P["fb2"]
    Zo = pn + D
    Y = np.maximum(Zo, 0)
    cache.update(X1=X1, Z1=Z1, A1=A1, X2=X2, Z2=Z2, A2=A2, X3=X3, Z3=Z3, A3=A3, s=s, pn=pn, f=f, Zh=Zh, Hh=Hh,
                 D=D, Zo=Zo, Y=Y, P=P)
    return Y * s[:, None], cache


def loss_and_grad(params, x, rows, target, nc):
    """L1 loss mean_b sum_c |y - target / s| over beams with s > 0, and its
    gradient with respect to the flat parameter vector (subgradient 0 at
    kinks)."""
    _, c = forward(params, x, rows, nc)
    P = c["P"]
    B = x.shape[0]
    s = c["s"]
    ok = s > 0
    y = np.where(ok[:, None], np.asarray(target, np.float64)[:, :nc] / np.where(ok, s, 1)[:, None], 0.0)
    e = c["Y"] - y
    loss = float(np.abs(e)[ok].sum() / B)
    dY = np.where(ok[:, None], np.sign(e), 0.0) / B
    dZo = dY * (c["Zo"] > 0)
    g = {}
    g["f2"] = dZo.T @ c["Hh"]
    g["fb2"] = dZo.sum(0)
    dH = dZo @ P["f2"]
    dZh = dH * (c["Zh"] > 0)
    g["f1"] = dZh.T @ c["f"]
    g["fb1"] = dZh.sum(0)
    df = dZh @ P["f1"]
    dA3 = df[:, :64 * C].reshape(B, 8, 8, C)
    dZ3 = dA3 * (c["Z3"] > 0)
    w3 = np.zeros((C, K2))
    w3[:, :306] = np.einsum("bhwo,bhwk->ok", dZ3, c["X3"])
    g["w3"], g["b3"] = w3, dZ3.sum((0, 1, 2))
    dX3 = dZ3 @ P["w3"][:, :306]
    dA2 = col2im(dX3, 16, 16, C + 2)[..., :C]
    dZ2 = dA2 * (c["Z2"] > 0)
    w2 = np.zeros((C, K2))
    w2[:, :306] = np.einsum("bhwo,bhwk->ok", dZ2, c["X2"])
    g["w2"], g["b2"] = w2, dZ2.sum((0, 1, 2))
    dX2 = dZ2 @ P["w2"][:, :306]
    dA1 = col2im(dX2, 32, 32, C + 2)[..., :C]
    dZ1 = dA1 * (c["Z1"] > 0)
    w1 = np.zeros((C, K1))
    w1[:, :18] = np.einsum("bhwo,bhwk->ok", dZ1, c["X1"])
    g["w1"], g["b1"] = w1, dZ1.sum((0, 1, 2))
    return loss, pack(g, nc)


def loss_only(params, x, rows, target, nc):
    tail, c = forward(params, x, rows, nc)
    s = c["s"]
    ok = s > 0
    y = np.where(ok[:, None], np.asarray(target, np.float64)[:, :nc] / np.where(ok, s, 1)[:, None], 0.0)
    return float(np.abs(c["Y"] - y)[ok].sum() / x.shape[0])
