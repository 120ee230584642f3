"""Pins of the warm-start network's oracle: the convolution against a library
correlation, and every gradient against central finite differences (rel 1e-6)."""

import numpy as np
import pytest

from oracle import net_oracle as NO


def test_conv_matches_library_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 6, 5, 7))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = NO.conv3d_same(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(ndimage.correlate(x[n, c], W[o, c], mode="constant", cval=0.0) for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=0, atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 2, 4, 5, 4))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    g = rng.standard_normal((2, 3, 4, 5, 4))
    dx, dW, db = NO.conv3d_same_backward(x, W, g)
    L = lambda x_, W_, b_: float(np.sum(NO.conv3d_same(x_, W_, b_) * g))
    h = 1e-6
    for arr, grad in ((x, dx), (W, dW), (b, db)):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]:
            old = arr[idx]
            arr[idx] = old + h
            lp = L(x, W, b)
            arr[idx] = old - h
            lm = L(x, W, b)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_network_gradients_finite_differences():
    rng = np.random.default_rng(2)
    params = NO.init_params(3)
    x = rng.standard_normal((2, 2, 10, 10, 10))
    target = rng.standard_normal((2, 4, 8, 8, 8))
    mask = (rng.random((2, 4, 8, 8, 8)) < 0.7).astype(float)
    out, acts = NO.forward(params, x)
    _, dout = NO.loss(out, target, mask)
    grads = NO.backward(params, acts, dout)

    def total():
        o, _ = NO.forward(params, x)
        return NO.loss(o, target, mask)[0]
    h = 1e-6
    for li in (0, 3):
        W, b = params[li]
        dW, db = grads[li]
        for idx in [tuple(rng.integers(0, s) for s in W.shape) for _ in range(6)]:
            old = W[idx]
            W[idx] = old + h
            lp = total()
            W[idx] = old - h
            lm = total()
            W[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - dW[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, dW[idx])
        j = int(rng.integers(0, b.shape[0]))
        old = b[j]
        b[j] = old + h
        lp = total()
        b[j] = old - h
        lm = total()
        b[j] = old
        assert abs((lp - lm) / (2 * h) - db[j]) <= 1e-6 * max(1.0, abs(db[j]))


def test_output_is_centre_and_padding_is_zero():
    params = NO.init_params(4)
    x = np.zeros((1, 2, 10, 10, 10))
    out, acts = NO.forward(params, x)
    assert out.shape == (1, 4, 8, 8, 8)
    # zero input: every activation is the bias chain, constant over the grid
    for a in acts[1:]:
        assert np.allclose(a, a[:, :, :1, :1, :1])
