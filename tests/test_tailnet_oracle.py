"""Pins of the FP64 tail-network statement (oracle/tailnet.py) to things other
than itself: the convolution against SciPy's 2-D correlation, col2im as the
exact adjoint of im2col, the gradient against central finite differences,
and the closed-form loss of a network whose correction layer is zero."""
import numpy as np
import pytest

from oracle import tailnet as TN

scipy_signal = pytest.importorskip("scipy.signal")

NC = 16


def random_case(seed, B=2, nc=NC):
    g = np.random.default_rng(seed)
    x = g.uniform(-1, 1.5, size=(B, 5440, 2))
    rows = np.zeros((B, nc + 4))
    rows[:, :nc] = g.uniform(0, 1, size=(B, nc))
    rows[:, nc + 3] = rows[:, :nc].sum(1)
    rows[:, nc + 1] = rows[:, nc + 3] * 1.5
    target = np.zeros_like(rows)
    target[:, :nc] = g.uniform(0, 1, size=(B, nc))
    lay, n = TN.layout(nc)
    p = np.zeros(n)
    for k, (o, s) in lay.items():
        fan = s[1] if len(s) == 2 else 1
        p[o:o + int(np.prod(s))] = g.uniform(-1, 1, size=int(np.prod(s))) * np.sqrt(3.0 / fan) * (0.3 if len(s) == 1 else 1)
    # padded conv columns are unused
    P = TN.unpack(p, nc)
    P["w1"][:, 18:] = 0
    P["w2"][:, 306:] = 0
    P["w3"][:, 306:] = 0
    return x, rows, target, TN.pack(P, nc)


def test_conv_matches_scipy_correlate():
    g = np.random.default_rng(1)
    a = g.normal(size=(1, 12, 10, 3))
    w = g.normal(size=(3, 3, 3))  # (ky, kx, c) of one output channel
    cols = TN.im2col(a)[0]        # [6, 5, 27]
    ours = cols @ np.array([w[t // 3, t % 3, c] for t in range(9) for c in range(3)])
    ref = np.zeros((6, 5))
    for c in range(3):
        padded = np.pad(a[0, :, :, c], 1)
        ref += scipy_signal.correlate2d(padded, w[:, :, c], mode="valid")[::2, ::2]
    np.testing.assert_allclose(ours, ref, rtol=1e-12, atol=1e-12)


def test_col2im_is_adjoint_of_im2col():
    g = np.random.default_rng(2)
    a = g.normal(size=(2, 16, 16, 5))
    d = g.normal(size=(2, 8, 8, 45))
    lhs = float((TN.im2col(a) * d).sum())
    rhs = float((a * TN.col2im(d, 16, 16, 5)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_gradient_matches_finite_differences():
    x, rows, target, p = random_case(3)
    loss, grad = TN.loss_and_grad(p, x, rows, target, NC)
    assert loss == pytest.approx(TN.loss_only(p, x, rows, target, NC), rel=1e-12)
    lay, _ = TN.layout(NC)
    g = np.random.default_rng(4)
    h = 1e-6
    for name, (o, s) in lay.items():
        size = int(np.prod(s))
        used = size
        if name in ("w1", "w2", "w3"):
            cols = 18 if name == "w1" else 306
            idx = [o + r * s[1] + c for r, c in zip(g.integers(0, s[0], 3), g.integers(0, cols, 3))]
        else:
            idx = list(o + g.integers(0, used, 3))
        for i in idx:
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (TN.loss_only(pp, x, rows, target, NC) - TN.loss_only(pm, x, rows, target, NC)) / (2 * h)
            assert grad[i] == pytest.approx(fd, rel=1e-4, abs=1e-7), (name, i)


def test_zero_correction_layer_returns_the_prior():
    x, rows, target, p = random_case(5)
    P = TN.unpack(p, NC)
    P["f2"][:] = 0
    P["fb2"][:] = 0
    p = TN.pack(P, NC)
    tail, _ = TN.forward(p, x, rows, NC)
    np.testing.assert_allclose(tail, rows[:, :NC], rtol=1e-12)
    s = np.maximum(rows[:, NC + 3], 0.1 * rows[:, NC + 1])
    expect = np.abs(rows[:, :NC] / s[:, None] - target[:, :NC] / s[:, None]).sum() / len(rows)
    assert TN.loss_only(p, x, rows, target, NC) == pytest.approx(expect, rel=1e-12)
