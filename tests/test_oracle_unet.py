"""Pins for oracle/unet.py: the convolution against scipy's correlate, the
pool / upsample adjoints, and every parameter gradient against central
finite differences in FP64."""

import numpy as np
import pytest
from scipy import signal

from oracle import unet


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv(x, w, b)
    for o in range(4):
        ref = sum(signal.correlate(x[c], w[o, c], mode="same") for c in range(3)) + b[o]
        assert np.allclose(y[o], ref, atol=1e-12)


def test_pool_and_up_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 6))
    g = rng.standard_normal((2, 4, 3))
    assert np.isclose(np.sum(unet.pool(x) * g), np.sum(x * unet.pool_backward(g)))
    h = rng.standard_normal((2, 8, 6))
    assert np.isclose(np.sum(unet.up(g) * h), np.sum(g * unet.up_backward(h)))


def test_gradients_by_finite_differences():
    c = (2, 3, 4)
    params = unet.init_params(3, cin=3, c=c)
    # nonzero biases so that every ReLU pattern is exercised
    rng = np.random.default_rng(4)
    params = {k: (w, rng.standard_normal(b.shape) * 0.1) for k, (w, b) in params.items()}
    xs = rng.standard_normal((2, 3, 8, 8))
    ts = rng.standard_normal((2, 1, 8, 8))
    loss, grads = unet.loss_and_grads(params, xs, ts)
    eps = 1e-6
    for name in unet.LAYERS:
        for which in (0, 1):
            arr = params[name][which]
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(3)]:
                saved = arr[idx]
                arr[idx] = saved + eps
                lp, _ = unet.loss_and_grads(params, xs, ts)
                arr[idx] = saved - eps
                lm, _ = unet.loss_and_grads(params, xs, ts)
                arr[idx] = saved
                fd = (lp - lm) / (2 * eps)
                an = grads[name][which][idx]
                assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, which, idx)


def test_adam_moves_against_the_gradient():
    params = unet.init_params(5, cin=3, c=(2, 3, 4))
    rng = np.random.default_rng(6)
    xs = rng.standard_normal((1, 3, 8, 8))
    ts = rng.standard_normal((1, 1, 8, 8))
    loss0, grads = unet.loss_and_grads(params, xs, ts)
    state = {}
    for _ in range(20):
        loss, grads = unet.loss_and_grads(params, xs, ts)
        params = unet.adam_step(params, grads, state, lr=1e-2)
    assert loss < loss0
