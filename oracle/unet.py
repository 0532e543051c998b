"""Reference U-Net of the learned preconditioner (NumPy, FP64 or FP32).

Not in the paper: the learned correction of the finite-difference
preconditioner is an addition (flexible CG with z = B r + s N(x), B the
paper's preconditioner of Sec. 3.1 or a diagonal scaling below alpha = 1).
This module is the plain definition the GPU kernels are checked against.

Network (channels c0, c1, c2 = 16, 32, 64 by default; every conv is 3 x 3
with zero padding and a bias; ReLU after every conv but the head):
    e0 = relu(conv(relu(conv(x))))               c0, H x W
    e1 = relu(conv(relu(conv(pool(e0)))))        c1, H/2
    b  = relu(conv(relu(conv(pool(e1)))))        c2, H/4
    d1 = relu(conv(relu(conv([up(b), e1]))))     c1, H/2
    d0 = relu(conv(relu(conv([up(d1), e0]))))    c0, H
    y  = head(d0)                                1 x 1 conv, 1 channel
pool = 2 x 2 average, up = 2 x 2 nearest, [a, b] = channel concatenation.
Parameters are a dict name -> (W, bias); conv weights W[cout, cin, 3, 3].

Loss: mean over the batch and the pixels of (y - t)^2.

BF16-operand variant (bf16_operands=True): the network as its tensor-core
convolutions define it.  Every 3 x 3 convolution multiplies the bfloat16
rounding (8 significant bits, round to nearest, ties to even) of its input
-- pooling, upsampling and concatenation applied first -- with the bfloat16
weights, and in the backward pass the product that forms the input gradient
takes the bfloat16 rounding of the upstream gradient.  Products are then
summed exactly (FP64 here); the weight gradients use the unrounded layer
input and upstream gradient.  The 1 x 1 head is not rounded.

Test infrastructure only.
"""

import numpy as np

LAYERS = ("e0a", "e0b", "e1a", "e1b", "ba", "bb", "d1a", "d1b", "d0a", "d0b", "head")


def layer_shapes(cin=3, c=(16, 32, 64)):
    c0, c1, c2 = c
    return {"e0a": (c0, cin, 3), "e0b": (c0, c0, 3), "e1a": (c1, c0, 3), "e1b": (c1, c1, 3),
            "ba": (c2, c1, 3), "bb": (c2, c2, 3), "d1a": (c1, c2 + c1, 3), "d1b": (c1, c1, 3),
            "d0a": (c0, c1 + c0, 3), "d0b": (c0, c0, 3), "head": (1, c0, 1)}


def init_params(seed, cin=3, c=(16, 32, 64), dtype=np.float64):
    """He-normal weights, zero biases, from numpy PCG64(seed) in LAYERS order."""
    rng = np.random.default_rng(seed)
    params = {}
    for name in LAYERS:
        co, ci, k = layer_shapes(cin, c)[name]
        std = np.sqrt(2.0 / (ci * k * k))
        params[name] = (rng.standard_normal((co, ci, k, k)).astype(dtype) * dtype(std),
                        np.zeros(co, dtype))
    return params


def bf16_round(a):
    """Round to the nearest value with an 8-bit significand (bfloat16),
    ties to even; zeros stay zero.  a = m 2^e with 1/2 <= |m| < 1, so the
    rounded value is rint(m 2^8) 2^(e-8)."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def conv(x, w, b):
    """'same' convolution (cross-correlation) of x[C, H, W] with w[O, C, k, k]."""
    o, c, k, _ = w.shape
    p = k // 2
    H, W = x.shape[1:]
    xp = np.pad(x, ((0, 0), (p, p), (p, p)))
    y = np.zeros((o, H, W), dtype=x.dtype)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + W]
            y += np.tensordot(w[:, :, dy, dx], patch, axes=(1, 0))
    return y + b[:, None, None]


def conv_backward(x, w, gy):
    """Gradients of conv: (dx, dw, db) for upstream gy[O, H, W]."""
    o, c, k, _ = w.shape
    p = k // 2
    H, W = x.shape[1:]
    xp = np.pad(x, ((0, 0), (p, p), (p, p)))
    dw = np.zeros_like(w)
    dxp = np.zeros_like(xp)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, dy:dy + H, dx:dx + W]
            dw[:, :, dy, dx] = np.tensordot(gy, patch, axes=((1, 2), (1, 2)))
            dxp[:, dy:dy + H, dx:dx + W] += np.tensordot(w[:, :, dy, dx], gy, axes=(0, 0))
    return dxp[:, p:p + H, p:p + W], dw, gy.sum(axis=(1, 2))


def pool(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(g):
    C, H, W = g.shape
    return g.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


def forward(params, x, keep=False, bf16_operands=False):
    """y = N(x) for one sample x[cin, H, W]; with keep=True also the
    activations needed by backward.  bf16_operands: the 3 x 3 convolutions
    take the bfloat16 rounding of their input (see the module docstring)."""
    acts = {}

    def cr(name, inp):
        w, b = params[name]
        q = bf16_round(inp) if bf16_operands and w.shape[-1] == 3 else inp
        z = conv(q, w, b)
        a = np.maximum(z, 0)
        acts[name] = (inp, z)
        return a

    e0 = cr("e0b", cr("e0a", x))
    e1 = cr("e1b", cr("e1a", pool(e0)))
    b = cr("bb", cr("ba", pool(e1)))
    c1 = b.shape[0]
    d1 = cr("d1b", cr("d1a", np.concatenate([up(b), e1])))
    d0 = cr("d0b", cr("d0a", np.concatenate([up(d1), e0])))
    y = conv(d0, *params["head"])
    acts["head"] = (d0, y)
    acts["_split"] = (c1, d1.shape[0])
    return (y, acts) if keep else y


def backward(params, acts, gy, bf16_operands=False):
    """Parameter gradients for upstream gradient gy[1, H, W].
    bf16_operands: the input gradient of each 3 x 3 convolution is formed
    from the bfloat16 rounding of its upstream gradient."""
    grads = {}

    def bk(name, g_out):
        inp, z = acts[name]
        w = params[name][0]
        gz = g_out * (z > 0) if name != "head" else g_out
        dx, dw, db = conv_backward(inp, w, gz)
        if bf16_operands and w.shape[-1] == 3:
            dx, _, _ = conv_backward(inp, w, bf16_round(gz))
        grads[name] = (dw, db)
        return dx

    c2, c1 = acts["_split"]
    g_d0 = bk("head", gy)
    g_cat0 = bk("d0a", bk("d0b", g_d0))
    g_up1, g_e0_skip = g_cat0[:c1], g_cat0[c1:]
    g_d1 = up_backward(g_up1)
    g_cat1 = bk("d1a", bk("d1b", g_d1))
    g_upb, g_e1_skip = g_cat1[:c2], g_cat1[c2:]
    g_b = up_backward(g_upb)
    g_e1 = pool_backward(bk("ba", bk("bb", g_b))) + g_e1_skip
    g_e0 = pool_backward(bk("e1a", bk("e1b", g_e1))) + g_e0_skip
    bk("e0a", bk("e0b", g_e0))
    return grads


def loss_and_grads(params, xs, ts, bf16_operands=False):
    """Mean squared error over a batch (xs[B, cin, H, W], ts[B, 1, H, W])
    and its parameter gradients (of the BF16-operand variant if asked)."""
    total = 0.0
    grads = None
    npix = ts[0].size
    for x, t in zip(xs, ts):
        y, acts = forward(params, x, keep=True, bf16_operands=bf16_operands)
        r = y - t
        total += float(np.sum(r * r)) / npix
        g = backward(params, acts, 2.0 * r / npix / len(xs), bf16_operands=bf16_operands)
        if grads is None:
            grads = g
        else:
            grads = {k: (grads[k][0] + g[k][0], grads[k][1] + g[k][1]) for k in grads}
    return total / len(xs), grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); state holds step count and moments."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for k, (w, b) in params.items():
        new = []
        for i, (p, g) in enumerate(((w, grads[k][0]), (b, grads[k][1]))):
            m = state.setdefault((k, i, "m"), np.zeros_like(p))
            v = state.setdefault((k, i, "v"), np.zeros_like(p))
            m[...] = b1 * m + (1 - b1) * g
            v[...] = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out[k] = tuple(new)
    return out
