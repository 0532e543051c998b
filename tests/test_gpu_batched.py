"""Batched solves (many problems of uneven size at once: one launch per pass
over all problems, CG iterations replayed as a CUDA graph, or with
FL_BATCH_PERSISTENT the inner CG iterations of each refinement step in one
persistent cooperative launch) against the FP64 oracle and against each
other."""

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


@pytest.mark.parametrize("launch", [0, _lib.FL_BATCH_PERSISTENT])
def test_batched_64_uneven_problems(launch):
    """64 problems, sides uniform in {96, 128, ..., 768}, alpha ~ U(0.3, 1.8),
    seeded Gaussian-mixture right-hand sides, to 1e-8; lockstep launches and
    the one persistent launch per refinement step."""
    sides = inputs.batch_sides(64, 7)
    alphas = inputs.alpha_draws(64, 8)
    plans, fd, fs = [], [], []
    for i, (n, a) in enumerate(zip(sides, alphas)):
        f = inputs.gaussian_mixture(n, 2, 16, 100 + i)
        fs.append(f)
        plans.append(Plan(2, (n, n), 1.0 / (n + 1), a))
        fd.append(torch.tensor(f, dtype=torch.float64, device="cuda:0").view(-1))
    us, infos = solve_batched(plans, fd, tol=1e-8,
                              mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO | launch)
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


def _batch_2d(sides, alphas, seed0):
    plans, fd, fs = [], [], []
    for i, (n, a) in enumerate(zip(sides, alphas)):
        f = inputs.gaussian_mixture(n, 2, 16, seed0 + i)
        fs.append(f)
        plans.append(Plan(2, (n, n), 1.0 / (n + 1), a))
        fd.append(torch.tensor(f, dtype=torch.float64, device="cuda:0").view(-1))
    return plans, fd, fs


@pytest.mark.parametrize("prec", [_lib.FL_PRECOND_AUTO, _lib.FL_PRECOND_FD, _lib.FL_PRECOND_NONE])
def test_persistent_launch_matches_lockstep(prec):
    """The persistent launch runs the same pass bodies as the lockstep
    launches (other row-pass CTA shapes, so other partial-sum groupings):
    both converge to 1e-8 in the oracle's FP64 residual, with iteration
    counts within two of each other and solutions that agree to the solve
    tolerance; one kernel launch per refinement step covers the CG."""
    sides = [96, 64, 160, 33, 128, 200, 17, 255]
    alphas = inputs.alpha_draws(len(sides), 5)
    plans, fd, fs = _batch_2d(sides, alphas, 300)
    lib = _lib.load()
    before = lib.fl_launch_count()
    us_p, inf_p = solve_batched(plans, fd, tol=1e-8,
                                mode=_lib.FL_MODE_MIXED | prec | _lib.FL_BATCH_PERSISTENT)
    torch.cuda.synchronize()
    launches_p = lib.fl_launch_count() - before
    before = lib.fl_launch_count()
    us_l, inf_l = solve_batched(plans, fd, tol=1e-8, mode=_lib.FL_MODE_MIXED | prec)
    torch.cuda.synchronize()
    launches_l = lib.fl_launch_count() - before
    for n, a, f, up, ul, ip, il in zip(sides, alphas, fs, us_p, us_l, inf_p, inf_l):
        assert ip["converged"] == 1 and il["converged"] == 1, (ip, il)
        assert abs(ip["iterations"] - il["iterations"]) <= 2, (n, a, ip, il)
        up = up.cpu().numpy().reshape(n, n)
        ul = ul.cpu().numpy().reshape(n, n)
        op = OPlan(2, n, 1.0 / (n + 1), a)
        res = np.linalg.norm(op.apply(up) - f) / np.linalg.norm(f)
        assert res <= 1.05e-8, (n, a, res)
        assert np.linalg.norm(up - ul) <= 1e-6 * np.linalg.norm(ul), (n, a)
    # per refinement step: start-up passes, the one CG launch, FP64 residual
    outer = max(i["outer_iterations"] for i in inf_p)
    its = max(i["iterations"] for i in inf_p)
    assert launches_p < launches_l
    assert launches_p <= 16 * (outer + 1), (launches_p, outer)
    assert launches_l >= its, (launches_l, its)


def test_persistent_launch_3d():
    shapes = [(24, 20, 28), (16, 16, 16), (33, 17, 9)]
    alphas = [0.6, 1.2, 1.7]
    plans, fd, fs = [], [], []
    for i, (n, a) in enumerate(zip(shapes, alphas)):
        f = inputs.gaussian_mixture(n, 3, 8, 500 + i)
        fs.append(f)
        plans.append(Plan(3, n, 1.0 / (max(n) + 1), a))
        fd.append(torch.tensor(f, dtype=torch.float64, device="cuda:0").view(-1))
    us_p, inf_p = solve_batched(plans, fd, tol=1e-8,
                                mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO | _lib.FL_BATCH_PERSISTENT)
    us_l, inf_l = solve_batched(plans, fd, tol=1e-8)
    torch.cuda.synchronize()
    for n, a, f, up, ul, ip, il in zip(shapes, alphas, fs, us_p, us_l, inf_p, inf_l):
        assert ip["converged"] == 1 and il["converged"] == 1, (ip, il)
        assert abs(ip["iterations"] - il["iterations"]) <= 2, (n, a, ip, il)
        up = up.cpu().numpy().reshape(n)
        op = OPlan(3, n, 1.0 / (max(n) + 1), a)
        res = np.linalg.norm(op.apply(up) - f) / np.linalg.norm(f)
        assert res <= 1.05e-8, (n, a, res)
        assert np.linalg.norm(up - ul.cpu().numpy().reshape(n)) <= 1e-6 * np.linalg.norm(up)


def test_grid_barrier_wait_is_bounded():
    """The persistent launch's grid barrier: with every CTA arriving it
    completes; with one arrival too few nobody releases it, every CTA gives
    up after its bounded wait (2 s) and the call reports FL_DEVICE_TIMEOUT;
    the context stays usable (a persistent batched solve after it
    converges)."""
    import time
    lib = _lib.load()
    assert lib.fl_check_grid_barrier(0) == _lib.FL_OK, _lib.last_error()
    t0 = time.perf_counter()
    st = lib.fl_check_grid_barrier(1)
    dt = time.perf_counter() - t0
    assert st == _lib.FL_DEVICE_TIMEOUT, _lib.last_error()
    assert "gave up" in _lib.last_error()
    assert 1.5 < dt < 60.0, dt
    assert lib.fl_check_grid_barrier(-1) == _lib.FL_INVALID_ARG
    plans, fd, fs = _batch_2d([48, 80], [0.7, 1.4], 600)
    _, infos = solve_batched(plans, fd, tol=1e-8,
                             mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO | _lib.FL_BATCH_PERSISTENT)
    assert all(i["converged"] == 1 for i in infos), infos


def test_lockstep_batch_in_the_256x8_row_shape():
    """Every plan in the 256 x 8 row shape: the lockstep batch runs its FP32
    row passes in that shape; it converges to 1e-8 in the oracle's residual
    with iteration counts within two of the default shape."""
    sides = [96, 160, 128, 200]
    alphas = [0.6, 1.1, 1.5, 0.9]
    plans, fd, fs = _batch_2d(sides, alphas, 700)
    _, inf0 = solve_batched(plans, fd, tol=1e-8)
    for p in plans:
        p.set_row_shape(1)
    us, inf1 = solve_batched(plans, fd, tol=1e-8)
    torch.cuda.synchronize()
    for n, a, f, u, i0, i1 in zip(sides, alphas, fs, us, inf0, inf1):
        assert i1["converged"] == 1, i1
        assert abs(i1["iterations"] - i0["iterations"]) <= 2, (n, a, i0, i1)
        op = OPlan(2, n, 1.0 / (n + 1), a)
        res = np.linalg.norm(op.apply(u.cpu().numpy().reshape(n, n)) - f) / np.linalg.norm(f)
        assert res <= 1.05e-8, (n, a, res)
