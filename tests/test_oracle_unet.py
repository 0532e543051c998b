"""Pins for oracle/unet.py: the convolution against scipy's correlate, the
pool / upsample adjoints, and every parameter gradient against central
finite differences in FP64."""

import math

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


# -- Adam (Kingma & Ba, Algorithm 1) pinned against values worked by hand ------
#
# With beta1 = 0.9, beta2 = 0.999 and the gradients g1 = 1/2, g2 = -1/4,
# g3 = 1 of one scalar parameter, the moments are, in exact arithmetic,
#   m1 = 1/20,   v1 = 1/4000,            m^1 = 1/2,      v^1 = 1/4
#   m2 = 1/50,   v2 = 1249/4000000,      m^2 = 2/19,     v^2 = 1249/7996
#   m3 = 59/500, v3 = 5247751/4e9,       m^3 = 118/271,  v^3 = 5247751/11988004
# (m_t = b1 m_{t-1} + (1-b1) g_t, v_t = b2 v_{t-1} + (1-b2) g_t^2,
# m^_t = m_t / (1 - b1^t), v^_t = v_t / (1 - b2^t)), and the parameter
# moves by -lr m^_t / (sqrt(v^_t) + eps) at step t.

HAND_M = (0.05, 0.02, 0.118)
HAND_V = (0.00025, 0.00031225, 0.00131193775)
HAND_MHAT = (1 / 2, 2 / 19, 118 / 271)
HAND_VHAT = (1 / 4, 1249 / 7996, 5247751 / 11988004)
HAND_G = (0.5, -0.25, 1.0)


def _scalar_params(p0):
    return {"s": (np.array([[[[p0]]]], dtype=np.float64), np.array([0.0]))}


def _adam_pin_failures(step):
    """Names of the hand-worked / closed-form Adam pins that `step` (an
    update with the signature of unet.adam_step) violates."""
    bad = []
    lr, eps = 1e-3, 1e-8
    # (a) three hand-worked steps: moments and parameter values
    params, state = _scalar_params(0.3), {}
    p = 0.3
    for t in range(3):
        grads = {"s": (np.array([[[[HAND_G[t]]]]]), np.array([0.0]))}
        params = step(params, grads, state, lr=lr, eps=eps)
        p -= lr * HAND_MHAT[t] / (math.sqrt(HAND_VHAT[t]) + eps)
        m = state.get(("s", 0, "m"))
        v = state.get(("s", 0, "v"))
        if m is None or v is None or abs(float(m.ravel()[0]) - HAND_M[t]) > 1e-15 \
                or abs(float(v.ravel()[0]) - HAND_V[t]) > 1e-15:
            bad.append("hand-worked moments")
            break
        if not abs(float(params["s"][0].ravel()[0]) - p) <= 1e-15:
            bad.append("hand-worked parameter")
            break
    # (b) a constant gradient g: the bias-corrected moments are exactly g and
    # g^2, so every step moves by lr g / (|g| + eps) -- t steps by t times that
    for g in (3.0, -0.02):
        params, state = _scalar_params(1.0), {}
        for _ in range(7):
            params = step(params, {"s": (np.array([[[[g]]]]), np.array([0.0]))}, state, lr=lr, eps=eps)
        want = 1.0 - 7 * lr * g / (abs(g) + eps)
        if not abs(float(params["s"][0].ravel()[0]) - want) <= 1e-14:
            bad.append("constant gradient")
            break
    # (c) eps is added to sqrt(v^): with |g| = eps the first step is lr / 2
    params = step(_scalar_params(0.0), {"s": (np.array([[[[eps]]]]), np.array([0.0]))}, {}, lr=lr,
                  eps=eps)
    if not abs(float(params["s"][0].ravel()[0]) + lr / 2) <= 1e-15:
        bad.append("epsilon placement")
    # (d) gradients +1 then -1: m2 = -(1-b1)^2, v2 = (1-b2^2), so
    # m^2 = -(1-b1)/(1+b1) = -1/19, v^2 = 1 and the second step is +lr/19
    params, state = _scalar_params(0.0), {}
    params = step(params, {"s": (np.array([[[[1.0]]]]), np.array([0.0]))}, state, lr=lr, eps=1e-300)
    p1 = float(params["s"][0].ravel()[0])
    params = step(params, {"s": (np.array([[[[-1.0]]]]), np.array([0.0]))}, state, lr=lr, eps=1e-300)
    if not (abs(p1 + lr) <= 1e-16 and abs(float(params["s"][0].ravel()[0]) - p1 - lr / 19) <= 1e-16):
        bad.append("alternating gradient")
    return bad


def test_adam_matches_hand_worked_steps():
    assert _adam_pin_failures(unet.adam_step) == []


def test_adam_updates_every_array_independently():
    """Weights and biases of several layers each follow their own moments:
    one step with gradient g moves every entry by lr g / (|g| + eps)."""
    params = unet.init_params(7, cin=3, c=(2, 3, 4))
    rng = np.random.default_rng(8)
    grads = {k: (rng.standard_normal(w.shape), rng.standard_normal(b.shape)) for k, (w, b) in params.items()}
    new = unet.adam_step(params, grads, {}, lr=1e-2, eps=1e-8)
    for k in params:
        for i in (0, 1):
            g = grads[k][i]
            assert np.allclose(params[k][i] - new[k][i], 1e-2 * g / (np.abs(g) + 1e-8), rtol=0,
                               atol=1e-16)


# planted mistakes: each variant of the update rule must fail one pin

def _adam_variant(no_bias_correction=False, eps_inside=False, swapped_betas=False,
                  lagged_count=False):
    def step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        with np.errstate(all="ignore"):
            return body(params, grads, state, lr, b1, b2, eps)

    def body(params, grads, state, lr, b1, b2, eps):
        if swapped_betas:
            b1, b2 = b2, b1
        t = state.get("t", 0) + (0 if lagged_count else 1)
        state["t"] = t + (1 if lagged_count else 0)
        out = {}
        for k, (w, b) in params.items():
            new = []
            for i, (p, g) in enumerate(((w, grads[k][0]), (b, grads[k][1]))):
                m = state.setdefault((k, i, "m"), np.zeros_like(p))
                v = state.setdefault((k, i, "v"), np.zeros_like(p))
                m[...] = b1 * m + (1 - b1) * g
                v[...] = b2 * v + (1 - b2) * g * g
                tt = max(t, 1)
                mh = m if no_bias_correction else m / (1 - b1 ** tt)
                vh = v if no_bias_correction else v / (1 - b2 ** tt)
                den = np.sqrt(vh + eps) if eps_inside else np.sqrt(vh) + eps
                new.append(p - lr * mh / den)
            out[k] = tuple(new)
        return out
    return step


@pytest.mark.parametrize("mistake", ["no_bias_correction", "eps_inside", "swapped_betas",
                                     "lagged_count"])
def test_planted_adam_mistakes_are_caught(mistake):
    assert _adam_pin_failures(_adam_variant(**{mistake: True})) != []


# -- the BF16-operand variant of the network ------------------------------------

def _bf16_by_bits(a):
    """bfloat16 as the upper 16 bits of the IEEE binary32 encoding, the lower
    16 bits rounded to nearest, ties to even (the format's definition)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lower = u & 0xFFFF
    upper = u >> 16
    up = (lower > 0x8000) | ((lower == 0x8000) & ((upper & 1) == 1))
    return ((upper + up) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_round_matches_the_bit_level_definition():
    rng = np.random.default_rng(30)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    assert np.array_equal(unet.bf16_round(x.astype(np.float64)), _bf16_by_bits(x))
    assert np.max(np.abs(unet.bf16_round(x) / x - 1)) <= 2.0 ** -8   # half a unit of 8 bits


def test_bf16_round_ties_and_representable_values():
    one = 1.0
    assert unet.bf16_round(one + 2.0 ** -8) == one                       # tie -> even (1.0)
    assert unet.bf16_round(one + 3 * 2.0 ** -8) == one + 2.0 ** -6       # tie -> even
    assert unet.bf16_round(-(one + 3 * 2.0 ** -8)) == -(one + 2.0 ** -6)
    exact = np.array([0.0, 1.0, -1.5, 255.0, 3 * 2.0 ** -20, 2.0 ** 100, -0.0078125])
    assert np.array_equal(unet.bf16_round(exact), exact)


def test_bf16_variant_rounds_exactly_the_3x3_operands(monkeypatch):
    """The variant inserts roundings and nothing else: with the rounding
    replaced by the identity it is the network itself, and the rounding is
    applied once per 3 x 3 convolution in the forward pass (its input) and
    once per 3 x 3 convolution in the backward pass (its upstream
    gradient) -- ten each, none for the 1 x 1 head."""
    params = unet.init_params(35, cin=3, c=(2, 3, 4))
    rng = np.random.default_rng(36)
    xs = rng.standard_normal((1, 3, 8, 8))
    ts = rng.standard_normal((1, 1, 8, 8))
    l0, g0 = unet.loss_and_grads(params, xs, ts)
    calls = []

    def ident(a):
        calls.append(np.shape(a))
        return np.asarray(a, dtype=np.float64)

    monkeypatch.setattr(unet, "bf16_round", ident)
    l1, g1 = unet.loss_and_grads(params, xs, ts, bf16_operands=True)
    assert l1 == l0
    for k in unet.LAYERS:
        assert np.array_equal(g1[k][0], g0[k][0]) and np.array_equal(g1[k][1], g0[k][1])
    assert len(calls) == 20
    conv3 = [k for k in unet.LAYERS if k != "head"]
    shapes = unet.layer_shapes(3, (2, 3, 4))
    # forward: the inputs, in layer order (channels = the layer's cin)
    assert [c[0] for c in calls[:10]] == [shapes[k][1] for k in conv3]
    # backward: the upstream gradients, in reverse layer order (cout)
    assert [c[0] for c in calls[10:]] == [shapes[k][0] for k in reversed(conv3)]


def test_bf16_variant_gradients_stay_close_to_the_exact_ones():
    params = unet.init_params(33, cin=3, c=(2, 3, 4))
    rng = np.random.default_rng(34)
    xs = rng.standard_normal((2, 3, 8, 8))
    ts = rng.standard_normal((2, 1, 8, 8))
    l0, g0 = unet.loss_and_grads(params, xs, ts)
    l1, g1 = unet.loss_and_grads(params, xs, ts, bf16_operands=True)
    assert l1 != l0 and abs(l1 - l0) <= 1e-2 * l0
    for k in unet.LAYERS:
        for i in (0, 1):
            assert np.linalg.norm(g1[k][i] - g0[k][i]) <= 5e-2 * np.linalg.norm(g0[k][i]) + 1e-12, k
