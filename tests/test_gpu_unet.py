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
        assert np.count_nonzero(d_ref) > 0.9 * d_ref.size
        err = np.abs(p1.astype(np.float64) - ref)
        bound = 1e-5 * np.abs(d_ref) + 2.0 ** -22 * np.abs(ref) + 1e-12
        assert np.all(err <= bound), (step, float(np.max(err / bound)))


def flatten64(params):
    return np.concatenate([np.ravel(a) for name in unet.LAYERS for a in params[name]])


@pytest.mark.parametrize("H", [64, 128])
def test_tensor_core_forward_matches_bf16_oracle(H):
    """tcgen05 forward (BF16 operands, FP32 accumulation in TMEM) against the
    oracle's BF16-operand network summed in FP64.  Bound 2e-4 (relative
    2-norm): FP32 accumulation error (~1e-6) plus the rare operand whose
    FP32 and FP64 values round to different BF16 neighbours (each such
    flip perturbs one operand by 2^-8 of its value; a few tens occur per
    forward); a wrong tap, channel or tile costs O(1)."""
    net, params = setup_net(H=H, seed=16, tensor_cores=True)
    x = np.random.default_rng(17).standard_normal((3, H, H)).astype(np.float32)
    y = net.forward(torch.tensor(x, device="cuda:0").view(-1)).cpu().numpy()
    net.check()
    ref = unet.forward(params, x.astype(np.float64), bf16_operands=True)[0].ravel()
    exact = unet.forward(params, x.astype(np.float64))[0].ravel()
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(f"H={H}: tcgen05 vs BF16 oracle {err:.2e}, BF16 oracle vs exact network "
          f"{np.linalg.norm(ref - exact) / np.linalg.norm(exact):.2e}")
    assert err <= 2e-4


def test_tensor_core_gradients_match_bf16_oracle():
    """A training step's loss and per-layer gradients on the tcgen05 path
    against the oracle's BF16-operand network (its input-gradient products
    take the BF16 upstream gradient; the weight gradients use the FP32
    values): loss to 1e-4, every layer's gradient to 1e-3 (relative
    2-norm, the forward bound grown by the backward pass)."""
    net, params = setup_net(seed=18, tensor_cores=True)
    rng = np.random.default_rng(19)
    xs = rng.standard_normal((2, 3, 64, 64)).astype(np.float32)
    ts = rng.standard_normal((2, 1, 64, 64)).astype(np.float32)
    loss = net.loss_grad(torch.tensor(xs, device="cuda:0"), torch.tensor(ts, device="cuda:0"))
    net.check()
    ref_loss, ref_grads = unet.loss_and_grads(params, xs.astype(np.float64), ts.astype(np.float64),
                                              bf16_operands=True)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    _, g = net.get_params(grads=True)
    gref = flatten(ref_grads)
    shapes = unet.layer_shapes()
    i = 0
    worst = 0.0
    for name in unet.LAYERS:
        co, ci, k = shapes[name]
        n = co * ci * k * k + co
        a, b = g[i:i + n].astype(np.float64), gref[i:i + n].astype(np.float64)
        e = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        worst = max(worst, e)
        assert e <= 1e-3, (name, e)
        i += n
    print(f"tcgen05 gradients vs BF16 oracle: worst layer {worst:.2e}")
