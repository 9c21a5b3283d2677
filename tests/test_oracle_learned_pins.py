"""Pins of the oracle's corrector building blocks (3x3x3 convolution, its
gradients, restriction).  These parts are not in the paper; each pin is a
mathematical identity of the definition: identity and shift kernels,
linearity, the adjoint identity <conv(x), g> = <x, conv^T(g)>, finite
differences of the weight and network gradients, and exactness of the
restriction on linear fields."""
import numpy as np
import pytest

import oracle


def rnd(shape, seed):
    return np.random.default_rng(seed).normal(size=shape)


def tap(dx, dy, dz):
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)


def test_identity_kernel():
    x = rnd((5, 6, 7, 3), 1)
    W = np.zeros((27, 3, 3))
    W[tap(0, 0, 0)] = np.eye(3)
    assert np.array_equal(oracle.conv3_fwd(x, W), x)


@pytest.mark.parametrize("d", [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                               (1, -1, 1)])
def test_shift_kernel_zero_padding(d):
    """A single 1 at tap (dx, dy, dz) reads x at p + (dx, dy, dz), zero
    outside the grid."""
    dx, dy, dz = d
    x = rnd((5, 6, 7, 2), 2)
    W = np.zeros((27, 2, 2))
    W[tap(dx, dy, dz)] = np.eye(2)
    y = oracle.conv3_fwd(x, W)
    pad = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    nz, ny, nx, _ = x.shape
    exp = pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    assert np.array_equal(y, exp)


def test_bias_and_linearity():
    x1, x2 = rnd((4, 5, 6, 3), 3), rnd((4, 5, 6, 3), 4)
    W = rnd((27, 3, 4), 5)
    b = rnd((4,), 6)
    y = oracle.conv3_fwd(x1, W, b)
    assert np.allclose(y, oracle.conv3_fwd(x1, W) + b, rtol=0, atol=1e-12)
    assert np.allclose(oracle.conv3_fwd(2 * x1 - x2, W), 2 * oracle.conv3_fwd(x1, W) - oracle.conv3_fwd(x2, W),
                       rtol=0, atol=1e-11)


def test_adjoint_identity():
    """<conv(x, W), g> = <x, conv_bwd_data(g, W)>: the input gradient is the
    exact adjoint of the forward map (catches a wrong tap flip or transpose)."""
    x = rnd((6, 5, 7, 3), 7)
    g = rnd((6, 5, 7, 4), 8)
    W = rnd((27, 3, 4), 9)
    lhs = np.sum(oracle.conv3_fwd(x, W) * g)
    rhs = np.sum(x * oracle.conv3_bwd_data(g, W))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_weight_gradient_finite_differences():
    """L(W, b) = sum(g * conv(x, W, b)) is linear, so central differences
    match the weight and bias gradients up to rounding."""
    x = rnd((4, 5, 6, 2), 10)
    g = rnd((4, 5, 6, 3), 11)
    W = rnd((27, 2, 3), 12)
    b = rnd((3,), 13)
    dW, db = oracle.conv3_bwd_weight(x, g)
    eps = 1e-3
    r = np.random.default_rng(14)
    for _ in range(12):
        t, c, o = int(r.integers(27)), int(r.integers(2)), int(r.integers(3))
        Wp, Wm = W.copy(), W.copy()
        Wp[t, c, o] += eps
        Wm[t, c, o] -= eps
        fd = (np.sum(g * oracle.conv3_fwd(x, Wp, b)) - np.sum(g * oracle.conv3_fwd(x, Wm, b))) / (2 * eps)
        assert abs(fd - dW[t, c, o]) <= 1e-6 * max(1.0, abs(fd))
    for o in range(3):
        bp, bm = b.copy(), b.copy()
        bp[o] += eps
        bm[o] -= eps
        fd = (np.sum(g * oracle.conv3_fwd(x, W, bp)) - np.sum(g * oracle.conv3_fwd(x, W, bm))) / (2 * eps)
        assert abs(fd - db[o]) <= 1e-6 * max(1.0, abs(fd))


def test_network_gradient_finite_differences():
    """The 4-layer corrector (3 -> 8 -> 8 -> 8 -> 1 channels here, ReLU between):
    backpropagated gradients of L = sum(r * z4) against central differences."""
    x = rnd((4, 4, 5, 3), 20)
    r = np.random.default_rng(21)
    chans = [3, 8, 8, 8, 1]
    params = [(r.normal(size=(27, chans[k], chans[k + 1])) * 0.3, r.normal(size=chans[k + 1]) * 0.1)
              for k in range(4)]
    rr = rnd((4, 4, 5, 1), 22)

    def loss(ps):
        return float(np.sum(rr * oracle.cnn_forward(x, ps)[-1]))

    acts = oracle.cnn_forward(x, params)
    grads = oracle.cnn_backward(x, params, acts, rr)
    eps = 1e-5
    for k in range(4):
        for _ in range(4):
            t = int(r.integers(27))
            c = int(r.integers(chans[k]))
            o = int(r.integers(chans[k + 1]))
            pp = [(W.copy(), b.copy()) for W, b in params]
            pm = [(W.copy(), b.copy()) for W, b in params]
            pp[k][0][t, c, o] += eps
            pm[k][0][t, c, o] -= eps
            fd = (loss(pp) - loss(pm)) / (2 * eps)
            assert abs(fd - grads[k][0][t, c, o]) <= 1e-6 * max(1.0, abs(fd)), (k, t, c, o)


def test_restriction_is_exact_on_linear_fields():
    """The mean of the fine points 4I+1, 4I+2 per axis is the trilinear value
    at the coarse cell centre (I + 1/2) * 4 h_f: exact for linear fields."""
    n, h = 32, 1.0 / 32
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = 0.3 * X - 1.7 * Y + 0.25 * Z + 0.125
    cc = (np.arange(n // 4) + 0.5) * (4 * h)
    Zc, Yc, Xc = np.meshgrid(cc, cc, cc, indexing="ij")
    assert np.allclose(oracle.restrict4(f), 0.3 * Xc - 1.7 * Yc + 0.25 * Zc + 0.125, rtol=0, atol=1e-14)
    assert np.array_equal(oracle.restrict4(np.full((8, 8, 8), 0.75)), np.full((2, 2, 2), 0.75))
