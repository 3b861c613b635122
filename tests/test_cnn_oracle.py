"""Pins of the CPU reference network (oracle/cnn_oracle.py): the convolution
against scipy's 2D correlation, the output's reduction to the masked linear
extrapolation when the last convolution is zero, and the back-propagated
gradients against central finite differences of the loss."""
import numpy as np
import pytest

from oracle import cnn_oracle as C


def test_conv3x3_matches_scipy_correlate2d():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    X = rng.normal(size=(7, 9, 3))
    Wm = rng.normal(size=(2, 27))
    b = np.array([0.3, -0.2])
    Y = C.conv3x3(X, Wm, b)
    for n in range(2):
        ref = np.full((7, 9), b[n])
        for c in range(3):
            k = Wm[n].reshape(9, 3)[:, c].reshape(3, 3)       # k[dy+1][dx+1]
            ref += scipy_signal.correlate2d(X[:, :, c], k, mode="same", boundary="fill")
        assert np.allclose(Y[:, :, n], ref, atol=1e-12)


def _features(rng, H, W):
    X = rng.normal(size=(H, W, 8))
    X[:, :, 7] = rng.random((H, W)) < 0.7          # activity mask
    return X


def test_zero_last_layer_gives_masked_linear_extrapolation():
    rng = np.random.default_rng(3)
    X = _features(rng, 5, 7)
    params = C.random_params(4)
    params[5] = (0 * params[5][0], 0 * params[5][1])
    _, out = C.forward(X, params)
    assert np.array_equal(out, np.where(X[:, :, 7] > 0, X[:, :, 6], 0.0))
    # no gradient reaches the network where the mask is off
    Xm = X.copy()
    Xm[:, :, 7] = 0
    _, grads, out = C.loss_and_grads(Xm, rng.normal(size=(5, 7)), C.random_params(4))
    assert not out.any() and all(not g.any() and not b.any() for g, b in grads)


@pytest.mark.parametrize("loss", ["mse", "l1"])
def test_gradients_match_finite_differences(loss):
    rng = np.random.default_rng(1)
    H = W = 6
    X = _features(rng, H, W)
    target = rng.normal(size=(H, W))
    params = C.random_params(2)
    value, grads, out = C.loss_and_grads(X, target, params, loss=loss)
    if loss == "l1":   # differentiable at these parameters: no residual near 0
        assert np.abs(out - target).min() > 1e-3
    eps = 1e-6
    for layer in range(6):
        Wm, b = params[layer]
        for _ in range(6):
            n = rng.integers(Wm.shape[0])
            k = rng.integers(Wm.shape[1])
            old = Wm[n, k]
            Wm[n, k] = old + eps
            lp = C.loss_and_grads(X, target, params, loss=loss)[0]
            Wm[n, k] = old - eps
            lm = C.loss_and_grads(X, target, params, loss=loss)[0]
            Wm[n, k] = old
            fd = (lp - lm) / (2 * eps)
            assert grads[layer][0][n, k] == pytest.approx(fd, rel=1e-5, abs=1e-9), (layer, n, k)
        n = rng.integers(b.shape[0])
        old = b[n]
        b[n] = old + eps
        lp = C.loss_and_grads(X, target, params, loss=loss)[0]
        b[n] = old - eps
        lm = C.loss_and_grads(X, target, params, loss=loss)[0]
        b[n] = old
        assert grads[layer][1][n] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-9), layer
