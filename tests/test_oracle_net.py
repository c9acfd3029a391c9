"""Pins of the warm-start network oracle (oracle/net.py) against what
mathematics and library routines fix: the convolution against
scipy.signal.correlate2d, gradients by central finite differences, Adam by its
closed form on constant gradients."""

import numpy as np
import pytest

from oracle import net as N

scipy_signal = pytest.importorskip("scipy.signal")


@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("H,W", [(7, 9), (8, 10), (15, 20)])
def test_conv_is_zero_padded_cross_correlation(stride, H, W):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, H, W))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = N.conv2d(x, w, b, stride)
    assert y.shape == (2, 4, N.out_size(H, stride), N.out_size(W, stride))
    for bi in range(2):
        for o in range(4):
            full = sum(scipy_signal.correlate2d(x[bi, c], w[o, c], mode="same", boundary="fill") for c in range(3))
            np.testing.assert_allclose(y[bi, o], full[::stride, ::stride] + b[o], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_backward_by_finite_differences(stride):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 7, 6))
    w = rng.standard_normal((5, 3, 3, 3))
    b = rng.standard_normal(5)
    dy = rng.standard_normal(N.conv2d(x, w, b, stride).shape)
    dx, dw, db = N.conv2d_backward(x, w, stride, dy)

    def f(x_, w_, b_):
        return float(np.sum(dy * N.conv2d(x_, w_, b_, stride)))

    h = 1e-6
    for arr, grad, name in ((x, dx, "x"), (w, dw, "w"), (b, db, "b")):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
            e = np.zeros_like(arr)
            e[idx] = h
            args_p = [x, w, b]
            args_m = [x, w, b]
            k = {"x": 0, "w": 1, "b": 2}[name]
            args_p[k] = arr + e
            args_m[k] = arr - e
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, grad[idx])


def test_network_shapes():
    p = N.init_params(0)
    y, _ = N.forward(p, np.zeros((3,) + N.IN_SHAPE))
    assert y.shape == (3,) + N.OUT_SHAPE


def test_mid_grey_input_gives_zero_through_a_network_without_biases():
    """The input is centred (I - 1/2): a network whose biases are all zero maps
    a uniform mid-grey quadruple to exactly zero whatever its weights (every
    layer is linear in its input up to ReLU, which keeps zero), and any other
    grey level to something non-zero."""
    p = [(w, np.zeros_like(b)) for w, b in N.init_params(7)]
    y, _ = N.forward(p, np.full((2,) + N.IN_SHAPE, 0.5))
    assert np.all(y == 0.0)
    y1, _ = N.forward(p, np.full((1,) + N.IN_SHAPE, 0.8))
    assert np.max(np.abs(y1)) > 0.0


def test_loss_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    p = N.init_params(4)
    # non-zero biases so every layer's bias gradient is exercised off zero
    p = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in p]
    imgs = rng.uniform(0, 1, (2,) + N.IN_SHAPE)
    target = rng.standard_normal((2,) + N.OUT_SHAPE)
    loss, grads = N.loss_and_grads(p, imgs, target)
    h = 1e-6
    for k in range(len(p)):
        for j in range(2):
            arr = p[k][j]
            for _ in range(3):
                idx = tuple(rng.integers(0, s) for s in arr.shape)

                def with_delta(d):
                    q = [list(t) for t in p]
                    a = arr.copy()
                    a[idx] += d
                    q[k][j] = a
                    return N.loss_and_grads([tuple(t) for t in q], imgs, target)[0]

                fd = (with_delta(h) - with_delta(-h)) / (2 * h)
                g = grads[k][j][idx]
                assert abs(fd - g) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (k, j, idx, fd, g)


def test_adam_closed_form_on_constant_gradients():
    """With a constant gradient g, m_hat = g and v_hat = g^2 at every step, so
    each step moves by lr * g / (|g| + eps)."""
    p = [(np.array([1.0, -2.0, 0.5]), np.array([0.0]))]
    g = [(np.array([0.3, -4.0, 1e-3]), np.array([2.0]))]
    st = N.adam_state(p)
    lr, eps = 0.01, 1e-8
    q = p
    for t in range(1, 4):
        q, st = N.adam_step(q, g, st, lr, eps=eps)
        for x0, x, gg in zip(p[0], q[0], g[0]):
            np.testing.assert_allclose(x, x0 - t * lr * gg / (np.abs(gg) + eps), rtol=1e-12, atol=1e-14)
    assert st[0] == 3


def test_relu_gates_the_gradient():
    """A layer whose pre-activations are all negative passes no gradient back."""
    p = N.init_params(5)
    w5, b5 = p[4]
    p[4] = (w5, np.full_like(b5, -1e6))
    imgs = np.random.default_rng(6).uniform(0, 1, (1,) + N.IN_SHAPE)
    _, grads = N.loss_and_grads(p, imgs, np.ones((1,) + N.OUT_SHAPE))
    for k in range(5):
        assert np.all(grads[k][0] == 0.0) and np.all(grads[k][1] == 0.0)
