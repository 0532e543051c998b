"""The U-Net kernels (forward, backward, Adam, checkpoints) against the NumPy
reference network of the oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet  # noqa: E402
from paper_1802_03770_gb300 import _lib  # noqa: E402
from paper_1802_03770_gb300.api import Net  # noqa: E402


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def flatten(params):
    out = []
    for name in unet.LAYERS:
        w, b = params[name]
        out += [np.ravel(w), np.ravel(b)]
    return np.concatenate(out).astype(np.float32)


def unflatten(flat, dtype=np.float64):
    shapes = unet.layer_shapes()
    params, i = {}, 0
    for name in unet.LAYERS:
        co, ci, k = shapes[name]
        nw = co * ci * k * k
        params[name] = (flat[i:i + nw].reshape(co, ci, k, k).astype(dtype),
                        flat[i + nw:i + nw + co].astype(dtype))
        i += nw + co
    return params


def setup_net(H=64, seed=1, tensor_cores=False):
    net = Net(H, H, seed=0)
    net.tensor_cores(tensor_cores)
    p = unet.init_params(seed, dtype=np.float64)
    rng = np.random.default_rng(seed + 1)
    p = {k: (w, rng.standard_normal(b.shape) * 0.05) for k, (w, b) in p.items()}
    flat = flatten(p)
    # weights as the kernels see them (BF16), biases FP32
    shapes = unet.layer_shapes()
    i = 0
    for name in unet.LAYERS:
        co, ci, k = shapes[name]
        nw = co * ci * k * k
        flat[i:i + nw] = bf16_round(flat[i:i + nw])
        i += nw + co
    net.set_params(flat)
    return net, unflatten(flat)


def test_forward_matches_oracle():
    net, params = setup_net()
    x = np.random.default_rng(3).standard_normal((3, 64, 64)).astype(np.float32)
    y = net.forward(torch.tensor(x, device="cuda:0").view(-1)).cpu().numpy()
    ref = unet.forward(params, x.astype(np.float64))[0]
    assert np.linalg.norm(y - ref.ravel()) <= 2e-5 * np.linalg.norm(ref)


def test_loss_and_gradients_match_oracle():
    net, params = setup_net(seed=5)
    rng = np.random.default_rng(6)
    xs = rng.standard_normal((2, 3, 64, 64)).astype(np.float32)
    ts = rng.standard_normal((2, 1, 64, 64)).astype(np.float32)
    loss = net.loss_grad(torch.tensor(xs, device="cuda:0"), torch.tensor(ts, device="cuda:0"))
    ref_loss, ref_grads = unet.loss_and_grads(params, xs.astype(np.float64), ts.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    _, g = net.get_params(grads=True)
    gref = flatten(ref_grads)
    shapes = unet.layer_shapes()
    i = 0
    for name in unet.LAYERS:
        co, ci, k = shapes[name]
        n = co * ci * k * k + co
        a, b = g[i:i + n], gref[i:i + n]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-12, name
        i += n


def test_adam_training_reduces_loss():
    net, _ = setup_net(seed=7)
    rng = np.random.default_rng(8)
    xs = torch.tensor(rng.standard_normal((2, 3, 64, 64)), dtype=torch.float32, device="cuda:0")
    ts = torch.tensor(rng.standard_normal((2, 1, 64, 64)) * 0.1, dtype=torch.float32, device="cuda:0")
    first = net.train_step(xs, ts, lr=1e-3)
    for _ in range(30):
        last = net.train_step(xs, ts, lr=1e-3)
    assert last < 0.5 * first


def test_checkpoint_roundtrip(tmp_path):
    net, _ = setup_net(seed=9)
    path = tmp_path / "net.bin"
    net.save(path)
    other = Net(64, 64, seed=123)
    other.load(path)
    assert np.array_equal(other.get_params(), net.get_params())
    raw = bytearray(path.read_bytes())
    raw[-1] ^= 0xFF
    path.write_bytes(bytes(raw))
    with pytest.raises(_lib.FracLapError, match="checksum"):
        other.load(path)


def test_tensor_core_forward_matches_cuda_core_forward():
    """tcgen05 path (BF16 activations): within 2e-2 of the FP32-activation
    path; the bound is BF16's 2^-9 unit roundoff on both GEMM operands,
    accumulated over ten 3 x 3 layers."""
    net, _ = setup_net(H=128, seed=11)
    x = torch.tensor(np.random.default_rng(12).standard_normal((3, 128, 128)), dtype=torch.float32,
                     device="cuda:0").view(-1)
    y32 = net.forward(x).cpu().numpy()
    net.tensor_cores(True)
    ytc = net.forward(x).cpu().numpy()
    net.check()
    assert np.linalg.norm(ytc - y32) <= 2e-2 * np.linalg.norm(y32)
    # and the training step runs on the tensor cores too
    xs = torch.tensor(np.random.default_rng(13).standard_normal((2, 3, 128, 128)), dtype=torch.float32,
                      device="cuda:0")
    ts = torch.zeros((2, 1, 128, 128), dtype=torch.float32, device="cuda:0")
    l0 = net.train_step(xs, ts, lr=1e-3)
    for _ in range(10):
        l1 = net.train_step(xs, ts, lr=1e-3)
    net.check()
    assert l1 < l0


def test_gpu_adam_matches_oracle_adam_step():
    """Two Adam steps of the GPU kernel against oracle.unet.adam_step, given
    the same parameters and the gradients the GPU formed.  The GPU works in
    FP32: per entry the bound is 1e-5 of the step plus two FP32 units of the
    parameter (the rounding of w - lr u)."""
    net, _ = setup_net(seed=14)
    rng = np.random.default_rng(15)
    state = {}
    lr = 1e-3
    for step in range(2):
        xs = torch.tensor(rng.standard_normal((2, 3, 64, 64)), dtype=torch.float32, device="cuda:0")
        ts = torch.tensor(rng.standard_normal((2, 1, 64, 64)), dtype=torch.float32, device="cuda:0")
        p0 = net.get_params().astype(np.float64)
        net.train_step(xs, ts, lr=lr)
        p1, g = net.get_params(grads=True)
        ref = flatten64(unet.adam_step(unflatten(p0), unflatten(g), state, lr=lr))
        d_ref = p0 - ref
        assert np.count_nonzero(d_ref) > 0.5 * d_ref.size   # not vacuous (dead ReLUs have g = 0)
        err = np.abs(p1.astype(np.float64) - ref)
        bound = 1e-5 * np.abs(d_ref) + 2.0 ** -22 * np.abs(ref) + 1e-12
        assert np.all(err <= bound), (step, float(np.max(err / bound)))


def flatten64(params):
    return np.concatenate([np.ravel(a) for name in unet.LAYERS for a in params[name]])


# Sources of each layer's input, as oracle.unet.forward assembles it:
# (tensor index, routing); tensor index 0 = the input features, l + 1 = the
# output of layer l (the numbering of Net.get_tensor).
SOURCES = {"e0a": [(0, "direct")], "e0b": [(1, "direct")], "e1a": [(2, "pool")],
           "e1b": [(3, "direct")], "ba": [(4, "pool")], "bb": [(5, "direct")],
           "d1a": [(6, "up"), (4, "direct")], "d1b": [(7, "direct")],
           "d0a": [(8, "up"), (2, "direct")], "d0b": [(9, "direct")], "head": [(10, "direct")]}
ROUTE = {"direct": lambda x: x, "pool": unet.pool, "up": unet.up}
ROUTE_BACK = {"direct": lambda g: g, "pool": unet.pool_backward, "up": unet.up_backward}


def _layer_input(acts, name):
    return np.concatenate([ROUTE[mode](acts[i]) for i, mode in SOURCES[name]])


@pytest.mark.parametrize("H", [64, 128])
def test_tensor_core_forward_layers_match_bf16_oracle(H):
    """Every layer of the tcgen05 forward against the oracle's BF16-operand
    convolution of the GPU's own input activations (pooling, upsampling and
    concatenation as the oracle assembles them, then BF16 rounding), summed
    in FP64: relative 2-norm <= 1e-5 per layer (FP32 accumulation of at most
    9 x 96 products, bias and ReLU; a wrong tap, channel, tile or rounding
    costs >= 1e-3).  End to end the two differ more (rounding boundaries
    crossed differently cascade through ten layers): bounded by 3e-3,
    against ~8e-3 between the BF16-operand and the exact network."""
    net, params = setup_net(H=H, seed=16, tensor_cores=True)
    x = np.random.default_rng(17).standard_normal((3, H, H)).astype(np.float32)
    y = net.forward(torch.tensor(x, device="cuda:0").view(-1)).cpu().numpy()
    net.check()
    acts = [net.get_tensor(i).astype(np.float64) for i in range(12)]
    assert np.array_equal(acts[0], x)
    worst = 0.0
    for li, name in enumerate(unet.LAYERS):
        w, b = params[name]
        inp = _layer_input(acts, name)
        q = unet.bf16_round(inp) if w.shape[-1] == 3 else inp
        z = unet.conv(q, w, b)
        ref = np.maximum(z, 0) if name != "head" else z
        e = np.linalg.norm(acts[li + 1] - ref) / np.linalg.norm(ref)
        worst = max(worst, e)
        assert e <= 1e-5, (name, e)
    ref_end = unet.forward(params, x.astype(np.float64), bf16_operands=True)[0].ravel()
    exact = unet.forward(params, x.astype(np.float64))[0].ravel()
    err = np.linalg.norm(y - ref_end) / np.linalg.norm(ref_end)
    print(f"H={H}: worst layer {worst:.2e}; end to end tcgen05 vs BF16 oracle {err:.2e}, BF16 "
          f"oracle vs exact network {np.linalg.norm(ref_end - exact) / np.linalg.norm(exact):.2e}")
    assert err <= 3e-3


def test_tensor_core_backward_layers_match_bf16_oracle():
    """One sample's backward pass on the tcgen05 path, layer by layer, from
    the GPU's own activations and upstream gradients: the loss gradient of
    the output, each layer's weight and bias gradients (FP32 on the CUDA
    cores: relative 2-norm <= 1e-4) and the gradient each tensor receives
    from its consumers (input-gradient products of BF16 upstream gradients
    on the tensor cores, routed back through pooling, upsampling and
    concatenation: <= 1e-5)."""
    H = 64
    net, params = setup_net(H=H, seed=18, tensor_cores=True)
    rng = np.random.default_rng(19)
    xs = rng.standard_normal((1, 3, H, H)).astype(np.float32)
    ts = rng.standard_normal((1, 1, H, H)).astype(np.float32)
    loss = net.loss_grad(torch.tensor(xs, device="cuda:0"), torch.tensor(ts, device="cuda:0"))
    net.check()
    acts = [net.get_tensor(i).astype(np.float64) for i in range(12)]
    grads = [net.get_tensor(i, grad=True).astype(np.float64) for i in range(12)]
    r = acts[11] - ts[0]
    assert loss == pytest.approx(float(np.mean(r * r)), rel=1e-6)
    assert np.linalg.norm(grads[11] - 2 * r / r.size) <= 1e-6 * np.linalg.norm(2 * r / r.size)
    _, g = net.get_params(grads=True)
    shapes = unet.layer_shapes()
    expect = [np.zeros_like(a) for a in acts]
    i = 0
    worst_w, worst_x = 0.0, 0.0
    for li, name in enumerate(unet.LAYERS):
        w, _ = params[name]
        co, ci, k = shapes[name]
        nw = co * ci * k * k
        o = li + 1
        gz = grads[o] * (acts[o] > 0) if name != "head" else grads[o]
        inp = _layer_input(acts, name)
        dx, dw, db = unet.conv_backward(inp, w, gz)
        ew = np.linalg.norm(g[i:i + nw] - dw.ravel()) / np.linalg.norm(dw)
        eb = np.linalg.norm(g[i + nw:i + nw + co] - db) / np.linalg.norm(db)
        worst_w = max(worst_w, ew, eb)
        assert ew <= 1e-4 and eb <= 1e-4, (name, ew, eb)
        i += nw + co
        if k == 3:
            dx, _, _ = unet.conv_backward(inp, w, unet.bf16_round(gz))
        c0 = 0
        for src, mode in SOURCES[name]:
            nc = acts[src].shape[0]
            expect[src] += ROUTE_BACK[mode](dx[c0:c0 + nc])
            c0 += nc
    for t in range(1, 11):
        e = np.linalg.norm(grads[t] - expect[t]) / np.linalg.norm(expect[t])
        worst_x = max(worst_x, e)
        assert e <= 1e-5, (t, e)
    print(f"tcgen05 backward vs BF16 oracle: weight gradients {worst_w:.2e}, "
          f"activation gradients {worst_x:.2e}")


def test_tensor_core_training_gradients_stay_near_the_bf16_oracle():
    """End to end over a batch of two, the tcgen05 training gradients and
    loss stay near the oracle's BF16-operand network (rounding boundaries
    crossed differently cascade, as in the forward): loss to 1e-3, every
    layer's gradient to 2e-2."""
    net, params = setup_net(seed=18, tensor_cores=True)
    rng = np.random.default_rng(19)
    xs = rng.standard_normal((2, 3, 64, 64)).astype(np.float32)
    ts = rng.standard_normal((2, 1, 64, 64)).astype(np.float32)
    loss = net.loss_grad(torch.tensor(xs, device="cuda:0"), torch.tensor(ts, device="cuda:0"))
    net.check()
    ref_loss, ref_grads = unet.loss_and_grads(params, xs.astype(np.float64), ts.astype(np.float64),
                                              bf16_operands=True)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    _, g = net.get_params(grads=True)
    gref = flatten(ref_grads)
    shapes = unet.layer_shapes()
    i = 0
    for name in unet.LAYERS:
        co, ci, k = shapes[name]
        n = co * ci * k * k + co
        a, b = g[i:i + n].astype(np.float64), gref[i:i + n].astype(np.float64)
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), name
        i += n
