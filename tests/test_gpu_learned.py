"""Flexible CG with the learned preconditioner, and the training pipeline."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.operator import Plan as OPlan  # noqa: E402
from paper_1802_03770_gb300 import _lib, inputs, learned  # noqa: E402
from paper_1802_03770_gb300.api import Net, Plan  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1802_03770_gb300", "weights", "unet512.bin")


@pytest.mark.parametrize("alpha", [0.7, 1.5])
def test_learned_solve_converges_with_untrained_network(alpha):
    """Flexible CG stays correct for any network: an untrained one either
    helps a little, hurts, or triggers the fallback to plain CG."""
    n = 64
    h = 1.0 / (n + 1)
    f = inputs.gaussian_mixture(n, 2, 8, 11)
    p = Plan(2, (n, n), h, alpha)
    net = Net(n, n, seed=3)
    p.attach_net(net)
    u, info = p.solve(torch.tensor(f, dtype=torch.float64, device="cuda:0"), tol=1e-8,
                      mode=_lib.FL_MODE_LEARNED | _lib.FL_PRECOND_AUTO)
    assert info["converged"] == 1
    op = OPlan(2, n, h, alpha)
    res = np.linalg.norm(op.apply(u.cpu().numpy()) - f) / np.linalg.norm(f)
    assert res <= 1.05e-8


def test_learned_mode_needs_a_network():
    p = Plan(2, (64, 64), 1.0 / 65, 1.0)
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.solve(torch.ones(64 * 64, dtype=torch.float64, device="cuda:0"),
                mode=_lib.FL_MODE_LEARNED)
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.attach_net(Net(128, 128))


def test_alpha_gate_falls_back_to_the_mixed_path():
    """With the plan's alpha band disabled, FL_MODE_LEARNED runs the plain
    FP32 preconditioned CG of FL_MODE_MIXED (same iterations, bitwise the
    same solution); with it enabled, the network runs again."""
    n, alpha = 64, 1.25
    f = torch.tensor(inputs.gaussian_mixture(n, 2, 8, 12), dtype=torch.float64, device="cuda:0")
    p = Plan(2, (n, n), 1.0 / (n + 1), alpha)
    net = Net(n, n, seed=3)
    p.attach_net(net)
    mixed = _lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO
    learn = _lib.FL_MODE_LEARNED | _lib.FL_PRECOND_AUTO
    u_m, i_m = p.solve(f, tol=1e-8, mode=mixed)
    u_l, i_l = p.solve(f, tol=1e-8, mode=learn)
    net.set_alpha_gate(0.3, 1.8, [1, 0, 1])          # bands of 0.5: alpha = 1.25 in the off band
    u_g, i_g = p.solve(f, tol=1e-8, mode=learn)
    assert i_g["iterations"] == i_m["iterations"]
    assert torch.equal(u_g, u_m)
    net.set_alpha_gate(0.3, 1.8, [0, 1, 0])
    u_g2, i_g2 = p.solve(f, tol=1e-8, mode=learn)
    assert i_g2["iterations"] == i_l["iterations"]
    assert torch.equal(u_g2, u_l)
    net.set_alpha_gate()                              # no gate: the network serves every alpha
    u_n, _ = p.solve(f, tol=1e-8, mode=learn)
    assert torch.equal(u_n, u_l)


def test_training_pipeline_reduces_loss_and_solves():
    net, hist = learned.train(n=64, pairs=96, batch=4, lr=2e-3, seed=5, pool=4, log_every=1)
    losses = [h[1] for h in hist]
    assert np.mean(losses[-4:]) < np.mean(losses[:4])
    ev = learned.evaluate(net, n=64, seeds=range(10000, 10004), pool=4)
    for row in ev:
        assert row["plain"]["converged"] and row["learned"]["converged"], row


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained 512 x 512 weights")
def test_trained_network_gain_on_held_out_seeds():
    """What the trained network gains (or loses) over plain CG, 512 x 512,
    held-out seeds: both converge to 1e-8; the gain is printed."""
    net = Net(512, 512)
    net.load(WEIGHTS)
    ev = learned.evaluate(net, n=512, seeds=range(10000, 10008), pool=8)
    plain = np.mean([r["plain"]["iterations"] for r in ev])
    lrn = np.mean([r["learned"]["iterations"] for r in ev])
    print(f"mean CG iterations: plain {plain:.1f}, learned {lrn:.1f}")
    for row in ev:
        assert row["plain"]["converged"] and row["learned"]["converged"], row


@pytest.mark.parametrize("alpha", [0.6, 1.4])
def test_training_pair_matches_oracle(alpha):
    """fl_net_training_pair against the pair formed from the oracle: r = f -
    M x (oracle apply), z0 = the FD-Laplacian box solve (DST-I) for alpha >=
    1, r / M_ii below, RMS scales, features [r/s_r, z0/s_z, alpha] and target
    (u* - x - z0)/s_z; FP32 outputs within FP32 rounding (1e-6 relative)."""
    from oracle import precond as oprec
    n = 40
    h = 1.0 / (n + 1)
    op = OPlan(2, n, h, alpha)
    plan = Plan(2, (n, n), h, alpha)
    f = inputs.gaussian_mixture(n, 2, 8, 71)
    rng = np.random.default_rng(72)
    u_star = rng.standard_normal((n, n))
    x = u_star + 0.1 * rng.standard_normal((n, n))
    dev = [torch.tensor(v, dtype=torch.float64, device="cuda:0").view(-1) for v in (f, u_star, x)]
    feat, target = plan.training_pair(*dev)
    torch.cuda.synchronize()
    feat = feat.cpu().numpy().astype(np.float64).reshape(3, n, n)
    target = target.cpu().numpy().astype(np.float64).reshape(n, n)
    r = f - op.apply(x).reshape(n, n)
    z0 = oprec.solve_box(op, r) if alpha >= 1.0 else r / op.entry(np.zeros(2))
    s_r = np.sqrt(np.mean(r * r))
    s_z = np.sqrt(np.mean(z0 * z0))
    refs = [r / s_r, z0 / s_z, np.full((n, n), alpha)]
    for k in range(3):
        assert np.linalg.norm(feat[k] - refs[k]) <= 1e-6 * np.linalg.norm(refs[k]), k
    ref_t = (u_star - x - z0) / s_z
    assert np.linalg.norm(target - ref_t) <= 1e-6 * np.linalg.norm(ref_t)


def test_training_pair_rejects_masked_plans():
    n = 16
    mask = np.ones((n, n), dtype=bool)
    mask[:4, :4] = False
    plan = Plan(2, (n, n), 1.0 / (n + 1), 1.2, mask=mask)
    z = torch.zeros(n * n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        plan.training_pair(z, z, z)
