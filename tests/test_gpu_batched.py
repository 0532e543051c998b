"""Batched solves (many problems of uneven size in lockstep, one launch per
pass, CG iterations replayed as a CUDA graph) against the FP64 oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.operator import Plan as OPlan  # noqa: E402
from paper_1802_03770_gb300 import _lib, inputs  # noqa: E402
from paper_1802_03770_gb300.api import Plan, solve_batched  # noqa: E402


def _problem(n, alpha, seed):
    f = inputs.gaussian_mixture(n, 2, 16, seed)
    return f, Plan(2, (n, n), 1.0 / (n + 1), alpha)


def test_batched_matches_single_solves():
    sides = [96, 64, 160, 33, 128, 200]
    alphas = inputs.alpha_draws(len(sides), 3)
    fs, plans = zip(*[_problem(n, a, 40 + i) for i, (n, a) in enumerate(zip(sides, alphas))])
    fd = [torch.tensor(f, dtype=torch.float64, device="cuda:0").view(-1) for f in fs]
    us, infos = solve_batched(list(plans), fd, tol=1e-8)
    torch.cuda.synchronize()
    for n, a, f, p, u, info in zip(sides, alphas, fs, plans, us, infos):
        assert info["converged"] == 1, info
        u = u.cpu().numpy().reshape(n, n)
        op = OPlan(2, n, 1.0 / (n + 1), a)
        res = np.linalg.norm(op.apply(u) - f) / np.linalg.norm(f)
        assert res <= 1.05e-8, (n, a, res)
        u1, _ = p.solve(torch.tensor(f, dtype=torch.float64, device="cuda:0"), tol=1e-10,
                        mode=_lib.FL_MODE_F64 | _lib.FL_PRECOND_AUTO)
        u1 = u1.cpu().numpy()
        assert np.linalg.norm(u - u1) <= 1e-6 * np.linalg.norm(u1)


def test_batched_64_uneven_problems():
    """64 problems, sides uniform in {96, 128, ..., 768}, alpha ~ U(0.3, 1.8),
    seeded Gaussian-mixture right-hand sides, to 1e-8."""
    sides = inputs.batch_sides(64, 7)
    alphas = inputs.alpha_draws(64, 8)
    plans, fd, fs = [], [], []
    for i, (n, a) in enumerate(zip(sides, alphas)):
        f = inputs.gaussian_mixture(n, 2, 16, 100 + i)
        fs.append(f)
        plans.append(Plan(2, (n, n), 1.0 / (n + 1), a))
        fd.append(torch.tensor(f, dtype=torch.float64, device="cuda:0").view(-1))
    us, infos = solve_batched(plans, fd, tol=1e-8)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    for i in rng.choice(64, 8, replace=False):
        n, a = sides[i], alphas[i]
        assert infos[i]["converged"] == 1, infos[i]
        op = OPlan(2, n, 1.0 / (n + 1), a)
        u = us[i].cpu().numpy().reshape(n, n)
        res = np.linalg.norm(op.apply(u) - fs[i]) / np.linalg.norm(fs[i])
        assert res <= 1.05e-8, (n, a, res)
    assert all(info["converged"] == 1 for info in infos)


def test_batched_rejects_mixed_dimensions_and_duplicates():
    a = Plan(2, (16, 16), 0.05, 1.0)
    b = Plan(3, (8, 8, 8), 0.1, 1.0)
    f2 = torch.zeros(256, dtype=torch.float64, device="cuda:0")
    f3 = torch.zeros(512, dtype=torch.float64, device="cuda:0")
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        solve_batched([a, b], [f2, f3])
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        solve_batched([a, a], [f2, f2])
