"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative 2-norms unless stated):
* FP64 apply / preconditioner: 1e-10 (the FP64 target of the build);
  FFT roundoff is about eps64 * log2(L) * cond, far below it.
* FP32 apply: 2e-5 for random fields (eps32 ~ 6e-8 times the log2 L ~ 11
  radix stages of the three passes times a safety factor of ~30 for the
  symbol's dynamic range), FP32 preconditioner: 2e-5.
* Solves: the FP64 relative residual computed by the oracle <= the requested
  tolerance (x 1.05 for the residual recomputed in another summation order),
  and the solution within cond-scaled distance of the oracle's.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import precond as opc  # noqa: E402
from oracle import solvers as osv  # noqa: E402
from oracle.operator import Plan as OPlan  # noqa: E402
from paper_1802_03770_gb300 import _lib, inputs  # noqa: E402
from paper_1802_03770_gb300.api import Plan  # noqa: E402

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def gpu(x, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


SHAPES = [
    (2, (64, 64)),        # the 64 x 64 solve case (L = 128)
    (2, (37, 53)),        # ragged, different L per axis
    (2, (1, 7)),          # degenerate axis
    (2, (3, 2)),
    (2, (130, 9)),        # rows far beyond one CTA, odd number of rows
    (3, (12, 9, 17)),
    (3, (5, 1, 6)),
    (3, (33, 20, 31)),
]


@pytest.mark.parametrize("d,n", SHAPES)
@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_apply_f64_matches_oracle(d, n, alpha):
    h = 1.0 / (max(n) + 1)
    op = OPlan(d, n, h, alpha)
    u = np.random.default_rng(10).standard_normal(n)
    y_ref = op.apply(u)
    p = Plan(d, n, h, alpha)
    y = host(p.apply(gpu(u)))
    assert rel(y, y_ref) <= 1e-10


@pytest.mark.parametrize("d,n", [(2, (64, 64)), (2, (37, 53)), (3, (12, 9, 17))])
def test_apply_direct_sum_small(d, n):
    """Against the O(N^2) definition, not only the oracle's FFT."""
    h = 0.03
    op = OPlan(d, n, h, 1.2)
    u = np.random.default_rng(11).standard_normal(n)
    y = host(Plan(d, n, h, 1.2).apply(gpu(u)))
    assert rel(y, op.apply_direct(u)) <= 1e-10


@pytest.mark.parametrize("d,n", [(2, (64, 64)), (2, (37, 53)), (3, (33, 20, 31)),
                                 (2, (1024, 1024)), (2, (1000, 333)), (3, (128, 128, 128))])
def test_apply_f32(d, n):
    """FP32 apply against the oracle, including the launch shapes of the
    full-size workloads (L = 2048: 128 x 16 row passes, 512 x 16 column
    passes, radix-16 stage plans, zero-half first stages; 3D L = 256)."""
    h = 1.0 / (max(n) + 1)
    op = OPlan(d, n, h, 1.3)
    rng = np.random.default_rng(12)
    u = rng.standard_normal(n)
    y = host(Plan(d, n, h, 1.3).apply(gpu(u, torch.float32)))
    assert rel(y, op.apply(u.astype(np.float32).astype(np.float64))) <= 2e-5


@pytest.mark.parametrize("d,n", [(2, (1, 4095)), (2, (3, 2500)), (2, (2100, 7)), (2, (1500, 40)),
                                 (2, (40, 1500))])
def test_apply_long_lines(d, n):
    """Padded lengths 4096 and 8192 (n_i up to 4095) along the row axis (the
    wide row-pass instantiations: one line per CTA of 256 or 512 threads)
    and along the strided axis (FP32 tiles of two or one column; the FP64
    column pass on 512 threads): FP64 to 1e-10, FP32 to 2e-5."""
    h = 1.0 / (max(n) + 1)
    op = OPlan(d, n, h, 1.3)
    u = np.random.default_rng(22).standard_normal(n)
    p = Plan(d, n, h, 1.3)
    assert rel(host(p.apply(gpu(u))), op.apply(u)) <= 1e-10
    u32 = u.astype(np.float32).astype(np.float64)
    assert rel(host(p.apply(gpu(u, torch.float32))), op.apply(u32)) <= 2e-5


def test_long_first_axis_rejects_the_fd_preconditioner():
    """The FD solve's tridiagonal pass holds columns of at most 1024 values:
    a plan with n_0 > 1024 solves with plain CG and refuses the FD
    preconditioner with FL_INVALID_ARG."""
    n = (1100, 8)
    h = 1.0 / 1101
    op = OPlan(2, n, h, 0.8)
    p = Plan(2, n, h, 0.8)
    f = np.random.default_rng(23).standard_normal(n)
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.precond(gpu(f))
    with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
        p.solve(gpu(f), mode=_lib.FL_MODE_F64 | _lib.FL_PRECOND_FD)
    u, info = p.solve(gpu(f), tol=1e-9, mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_NONE, maxit=3000)
    assert info["converged"] == 1
    assert rel(op.apply(host(u)), f) <= 1.05e-9


def test_apply_masked():
    n = (41, 30)
    rng = np.random.default_rng(13)
    mask = rng.random(n) < 0.8
    op = OPlan(2, n, 0.02, 1.1, mask=mask)
    u = rng.standard_normal(n)
    y = host(Plan(2, n, 0.02, 1.1, mask=mask).apply(gpu(u)))
    assert np.all(y[~mask] == 0.0)
    assert rel(y, op.apply(u)) <= 1e-10


def test_apply_is_deterministic():
    n = (96, 80)
    p = Plan(2, n, 0.01, 0.9)
    u = gpu(np.random.default_rng(14).standard_normal(n))
    a, b = host(p.apply(u)), host(p.apply(u))
    assert np.array_equal(a, b)


def test_plan_constants_match_oracle():
    for d, n, alpha in [(2, (64, 64), 1.0), (3, (10, 12, 14), 1.7), (2, (5, 9), 0.2)]:
        h = 1.0 / 65
        op = OPlan(d, n, h, alpha)
        desc = Plan(d, n, h, alpha).describe()
        assert desc["c_alpha_d"] == pytest.approx(op.C, rel=1e-13)
        assert desc["lattice_zeta"] == pytest.approx(op.A1 * h ** (d + alpha), rel=1e-12)
        assert desc["window_corr"] == pytest.approx((op.A2 + op.A3) * h ** (d + alpha - 2), rel=1e-11)
        assert desc["kernel0"] == pytest.approx(float(op.entry(np.zeros(d))), rel=1e-11)
        assert all(L >= 2 * v - 1 for L, v in zip(desc["fft_len"], n))


@pytest.mark.parametrize("d,n", [(2, (64, 64)), (2, (37, 53)), (2, (1, 6)), (3, (12, 9, 17)),
                                 (3, (33, 20, 31)), (2, (1024, 1024)), (2, (1000, 333)),
                                 (3, (97, 8, 40))])
@pytest.mark.parametrize("shift,scale", [(0.0, 1.0), (1.0, 2e-3)])
def test_precond_matches_oracle(d, n, shift, scale):
    h = 1.0 / (max(n) + 1)
    op = OPlan(d, n, h, 1.4)
    r = np.random.default_rng(15).standard_normal(n)
    z_ref = opc.solve_box(op, r, shift, scale)
    p = Plan(d, n, h, 1.4)
    z = host(p.precond(gpu(r), shift, scale))
    assert rel(z, z_ref) <= 1e-10
    z32 = host(p.precond(gpu(r, torch.float32), shift, scale))
    assert rel(z32, z_ref) <= 2e-5


def test_solve_64_f64_matches_dense_lu():
    """64 x 64, alpha = 1, 8 Gaussians, FP64 PCG to 1e-10; dense LU check."""
    n = 64
    h = 1.0 / (n + 1)
    f = inputs.gaussian_mixture(n, 2, 8, 0, 0.05, 0.2)
    op = OPlan(2, n, h, 1.0)
    u_lu = np.linalg.solve(op.dense_matrix(), f.ravel()).reshape(n, n)
    p = Plan(2, (n, n), h, 1.0)
    u, info = p.solve(gpu(f), tol=1e-10, mode=_lib.FL_MODE_F64)
    u = host(u)
    assert info["converged"] == 1 and info["iterations"] > 5
    assert rel(op.apply(u), f) <= 1.05e-10
    assert rel(u, u_lu) <= 1e-8


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
@pytest.mark.parametrize("mode", [_lib.FL_MODE_F64, _lib.FL_MODE_MIXED])
def test_solve_255(alpha, mode):
    n = 255
    h = 1.0 / (n + 1)
    f = inputs.gaussian_mixture(n, 2, 32, 1)
    op = OPlan(2, n, h, alpha)
    p = Plan(2, (n, n), h, alpha)
    u, info = p.solve(gpu(f), tol=1e-8, mode=mode | _lib.FL_PRECOND_AUTO, maxit=2000)
    u = host(u)
    assert info["converged"] == 1
    assert rel(op.apply(u), f) <= 1.05e-8
    u_ref, _, ok, _ = osv.solve_elliptic(op, f, 1e-12, 4000, alpha >= 1.0)
    assert ok
    assert rel(u, u_ref) <= 1e-5


def test_solve_host_arrays():
    n = 48
    f = inputs.gaussian_mixture(n, 2, 8, 2)
    op = OPlan(2, n, 1.0 / (n + 1), 1.25)
    p = Plan(2, (n, n), 1.0 / (n + 1), 1.25)
    u, info = p.solve_host(f, tol=1e-9)
    assert info["converged"] == 1
    assert rel(op.apply(u), f) <= 1.05e-9


def test_solve_masked_plain_cg():
    n = (40, 40)
    ax = np.linspace(-1, 1, 40)
    X, Y = np.meshgrid(ax, ax, indexing="ij")
    mask = X ** 2 + Y ** 2 < 0.9
    op = OPlan(2, n, 0.05, 0.75, mask=mask)
    f = np.where(mask, 1.0, 0.0)
    p = Plan(2, n, 0.05, 0.75, mask=mask)
    u, info = p.solve(gpu(f), tol=1e-9, mode=_lib.FL_MODE_F64 | _lib.FL_PRECOND_NONE)
    u = host(u)
    assert np.all(u[~mask] == 0.0)
    assert rel(op.apply(u), f) <= 1.05e-9


def test_precond_rejects_nonpositive_scale():
    p = Plan(2, (16, 16), 0.05, 1.5)
    r = gpu(np.ones((16, 16)))
    for shift, scale in [(1.0, 0.0), (0.0, -1.0), (-1.0, 1.0)]:
        with pytest.raises(_lib.FracLapError, match="INVALID_ARG"):
            p.precond(r, shift, scale)


def _l_shape(n):
    ax = [np.linspace(-1, 1, k) for k in n]
    G = np.meshgrid(*ax, indexing="ij")
    return ~np.logical_and.reduce([g > 0 for g in G])


@pytest.mark.parametrize("d,n", [(2, (48, 40)), (3, (12, 10, 14)), (2, (127, 127))])
@pytest.mark.parametrize("shift,scale", [(0.0, 1.0), (1.0, 2e-3)])
def test_precond_masked_matches_oracle(d, n, shift, scale):
    """Occluded domain: the FD operator on Omega with Dirichlet conditions
    on the hole (the paper's preconditioner, Sec. 4.4), applied by the box
    solve and the hole boundary's capacitance matrix, against the oracle's
    sparse direct solve: FP64 to 1e-10; FP32 box solves (the interface
    system in FP64) to 1e-4 -- the capacitance solve amplifies the FP32
    box solves' rounding by the conditioning of the interface system."""
    mask = _l_shape(n)
    h = 1.0 / (max(n) + 1)
    op = OPlan(d, n, h, 1.4, mask=mask)
    r = np.random.default_rng(21).standard_normal(n)
    z_ref = opc.solve_domain(op, r, shift, scale)
    p = Plan(d, n, h, 1.4, mask=mask)
    z = host(p.precond(gpu(r), shift, scale))
    assert np.all(z[~mask] == 0.0)
    e64 = rel(z, z_ref)
    z32 = host(p.precond(gpu(r, torch.float32), shift, scale))
    e32 = rel(z32, z_ref)
    print(f"masked precond {n}: FP64 {e64:.1e}, FP32 {e32:.1e}")
    assert e64 <= 1e-10
    assert e32 <= 1e-4


@pytest.mark.parametrize("mode", [_lib.FL_MODE_F64, _lib.FL_MODE_MIXED])
def test_solve_masked_preconditioned(mode):
    """L-shaped domain, alpha = 1.5: the FD operator on Omega, the restricted
    box solve and plain CG converge to the same solution; the paper's
    preconditioner takes the fewest iterations."""
    n = (64, 64)
    mask = _l_shape(n)
    h = 1.0 / 65
    op = OPlan(2, n, h, 1.5, mask=mask)
    f = np.where(mask, inputs.gaussian_mixture(64, 2, 8, 3), 0.0)
    p = Plan(2, n, h, 1.5, mask=mask)
    its = {}
    sols = {}
    for name, pm in (("domain", _lib.FL_PRECOND_FD), ("box", _lib.FL_PRECOND_BOX),
                     ("plain", _lib.FL_PRECOND_NONE)):
        u, info = p.solve(gpu(f), tol=1e-9, mode=mode | pm)
        u = host(u)
        assert info["converged"] == 1 and np.all(u[~mask] == 0.0)
        assert rel(op.apply(u), f) <= 1.05e-9
        its[name] = info["iterations"]
        sols[name] = u
    assert rel(sols["domain"], sols["plain"]) <= 1e-6 and rel(sols["box"], sols["plain"]) <= 1e-6
    print(f"L-shape 64^2, alpha 1.5: iterations {its}")
    assert its["domain"] < its["box"] < its["plain"]


def _octagon(n):
    i = np.arange(1, n)
    a = np.minimum(i, n - i)
    return (a[:, None] + a[None, :]) > n // 4


def _l_shape_paper(n):
    m = n - 1
    mask = np.ones((m, m), dtype=bool)
    mask[m - n // 2:, m - n // 2:] = False
    return mask


@pytest.mark.parametrize("shape", ["lshape", "octagon"])
def test_occluded_tables_first_rows_on_gpu(shape):
    """Tables tab:L2 and tab:octagon2, n = 128 and 256 (N = 12033 / 48641 and
    14145 / 56961), alpha = 1.75, f = 1 on Omega, FP64 CG with the FD
    operator on Omega: the oracle's counts (10 / 14 and 12 / 16, which are
    the print's for n = 128 and within one of it for n = 256)."""
    for n, want in ((128, (10, 14)), (256, (12, 16))):
        mask = _l_shape_paper(n) if shape == "lshape" else _octagon(n)
        p = Plan(2, mask.shape, 1.0 / n, 1.75, mask=mask)
        f = gpu(np.where(mask, 1.0, 0.0))
        got = tuple(p.solve(f, tol=tol, mode=_lib.FL_MODE_F64 | _lib.FL_PRECOND_FD,
                            maxit=1000)[1]["iterations"] for tol in (1e-6, 1e-9))
        print(f"{shape} n = {n} (N = {int(mask.sum())}): {got}")
        assert got == want, (shape, n, got)


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_consecutive_time_steps_reuse_m_u(theta):
    """Three mixed steps u0 -> u1 -> u2 -> u3 (the second and third start from
    the M u the previous step's last FP64 residual left), then a step from an
    array changed in place (its hash differs: M u is recomputed) -- all
    against the oracle's steps."""
    n = (20, 18, 16)
    h = 1.0 / 21
    op = OPlan(3, n, h, 1.5)
    u0 = inputs.gaussian_mixture(20, 3, 16, 4, 0.05, 0.15)[:, :18, :16].copy()
    dt = 1e-3
    p = Plan(3, n, h, 1.5)
    a, b = gpu(u0), torch.empty(int(np.prod(n)), dtype=torch.float64, device="cuda")
    ref = u0
    for _ in range(3):
        ref, _, ok, _ = osv.theta_step(op, ref, dt, theta, None, None, tol=1e-13)
        assert ok
        _, info = p.time_step(a, dt, theta, out=b, tol=1e-10, mode=_lib.FL_MODE_MIXED)
        assert info["converged"] == 1
        assert rel(host(b).reshape(n), ref) <= 1e-9
        a, b = b, a
    # change the current state in place: the cached M u must not be used
    a.mul_(0.5)
    ref, _, ok, _ = osv.theta_step(op, 0.5 * ref, dt, theta, None, None, tol=1e-13)
    _, info = p.time_step(a, dt, theta, out=b, tol=1e-10, mode=_lib.FL_MODE_MIXED)
    assert info["converged"] == 1
    assert rel(host(b).reshape(n), ref) <= 1e-9


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("mode", [_lib.FL_MODE_F64, _lib.FL_MODE_MIXED])
def test_time_step_3d(theta, mode):
    n = 24
    h = 1.0 / (n + 1)
    op = OPlan(3, n, h, 1.5)
    u0 = inputs.gaussian_mixture(n, 3, 16, 4, 0.05, 0.15)
    f0 = inputs.gaussian_mixture(n, 3, 4, 5)
    f1 = inputs.gaussian_mixture(n, 3, 4, 6)
    dt = 1e-3
    u_ref, _, ok, _ = osv.theta_step(op, u0, dt, theta, f0, f1, tol=1e-13)
    assert ok
    p = Plan(3, (n, n, n), h, 1.5)
    u, info = p.time_step(gpu(u0), dt, theta, gpu(f0), gpu(f1), tol=1e-10, mode=mode)
    assert info["converged"] == 1
    assert rel(host(u), u_ref) <= 1e-9


def test_breakdown_and_cap_statuses():
    n = 32
    p = Plan(2, (n, n), 1.0 / (n + 1), 1.5)
    f = gpu(inputs.gaussian_mixture(n, 2, 8, 7))
    u, info = p.solve(f, tol=1e-12, maxit=2, mode=_lib.FL_MODE_F64, raise_on_fail=False)
    assert info["status"] == _lib.FL_NOT_CONVERGED and info["converged"] == 0
    nan = gpu(np.full((n, n), np.nan))
    u, info = p.solve(nan, tol=1e-8, mode=_lib.FL_MODE_F64, raise_on_fail=False)
    assert info["status"] in (_lib.FL_BREAKDOWN, _lib.FL_NOT_CONVERGED)
    zero = gpu(np.zeros((n, n)))
    u, info = p.solve(zero, tol=1e-8, mode=_lib.FL_MODE_MIXED)
    assert info["converged"] == 1 and float(u.abs().max()) == 0.0


# -- full sizes ---------------------------------------------------------------

def test_full_size_2d_1024_apply_and_mixed_solve():
    """1024 x 1024 (2048^2 padded FFT), alpha = 1.5, 32 Gaussians."""
    n = 1024
    h = 1.0 / (n + 1)
    f = inputs.gaussian_mixture(n, 2, 32, 0)
    op = OPlan(2, n, h, 1.5)
    p = Plan(2, (n, n), h, 1.5)
    y = host(p.apply(gpu(f)))
    assert rel(y, op.apply(f)) <= 1e-10
    u, info = p.solve(gpu(f), tol=1e-8, mode=_lib.FL_MODE_MIXED)
    assert info["converged"] == 1
    assert rel(op.apply(host(u)), f) <= 1.05e-8


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_full_size_2d_1024_mixed_solution_error(alpha):
    """The 1024 x 1024 workload's mixed solves (FP32 inner CG + FP64
    refinement to 1e-8, the bench's preconditioner choice) against a tight
    FP64 oracle solve (1e-12): the FP64 residual recomputed by the oracle
    and the solution's relative error, printed.  The error is bounded by
    cond(M) times the residual; cond(M) ~ (n+1)^alpha here, at most ~3e4."""
    n = 1024
    h = 1.0 / (n + 1)
    f = inputs.gaussian_mixture(n, 2, 32, 0)
    op = OPlan(2, n, h, alpha)
    p = Plan(2, (n, n), h, alpha)
    u, info = p.solve(gpu(f), tol=1e-8, mode=_lib.FL_MODE_MIXED | _lib.FL_PRECOND_AUTO, maxit=2000)
    u = host(u)
    assert info["converged"] == 1
    res = rel(op.apply(u), f)
    u_ref, its, ok, _ = osv.solve_elliptic(op, f, 1e-12, 4000, alpha >= 1.0)
    assert ok
    err = rel(u, u_ref)
    print(f"1024^2 alpha={alpha}: mixed {info['iterations']} inner its, {info['outer_iterations']} "
          f"refinements, oracle residual {res:.3e}, error vs FP64 oracle {err:.3e} "
          f"(oracle {its} its to 1e-12)")
    assert res <= 1.05e-8
    assert err <= 3e4 * 1.05e-8


def _direct_samples(op, u, idx):
    """(M u)_i at sample points i by the plain definition (O(N) each)."""
    pts = op.points()
    vals = u[tuple(pts.T)]
    out = []
    for i in idx:
        k = op.entry(pts - np.asarray(i)[None, :])
        out.append(float(np.dot(k, vals)))
    return np.array(out)


def test_full_size_3d_256_apply_samples():
    """256^3 (512^3 padded FFT), alpha = 1.5: sampled outputs by direct sum."""
    n = 256
    h = 1.0 / (n + 1)
    u = inputs.gaussian_mixture(n, 3, 16, 3, 0.05, 0.15)
    op = OPlan(3, n, h, 1.5)
    p = Plan(3, (n, n, n), h, 1.5)
    y = host(p.apply(gpu(u)))
    rng = np.random.default_rng(16)
    idx = [tuple(rng.integers(0, n, 3)) for _ in range(6)] + [(0, 0, 0), (255, 255, 255), (128, 0, 77)]
    ref = _direct_samples(op, u, idx)
    got = np.array([y[i] for i in idx])
    scale = np.abs(y).max()
    assert np.max(np.abs(got - ref)) <= 1e-10 * scale
    # the FP32 apply at the same points, against the definition applied to
    # the FP32-rounded input
    y32 = host(p.apply(gpu(u, torch.float32))).astype(np.float64)
    ref32 = _direct_samples(op, u.astype(np.float32).astype(np.float64), idx)
    got32 = np.array([y32[i] for i in idx])
    assert np.max(np.abs(got32 - ref32)) <= 2e-5 * scale


def test_table_td_its_on_gpu(golden):
    """Table tab:td_its on the GPU: one Crank-Nicolson system with random RHS
    from a zero start (u_prev = 0, f_prev = f_next = b / dt), FP64 CG with the
    I + dt/2 C h^d L preconditioner: the paper's preconditioned counts."""
    for d, n, alpha, its_p, _ in golden("table_td_its.txt"):
        d, n = int(d), int(n)
        if d == 3:
            continue
        dt = 1.0 / (n + 1)
        b = inputs.random_field(n, d, 0)
        p = Plan(d, (n,) * d, 1.0 / (n + 1), alpha)
        zero = gpu(np.zeros((n,) * d))
        f = gpu(b / dt)
        _, info = p.time_step(zero, dt, 0.5, f, f, tol=1e-9, mode=_lib.FL_MODE_F64)
        assert info["iterations"] == int(its_p), (alpha, info)


def test_table_3d_its_on_gpu(golden):
    """Table tab:3D_its preconditioned counts (f = 1, 31^3, 1e-9) on the GPU."""
    for n, alpha, its_p, _ in golden("table_3d_its.txt"):
        n = int(n)
        p = Plan(3, (n, n, n), 1.0 / (n + 1), alpha)
        _, info = p.solve(gpu(np.ones((n, n, n))), tol=1e-9, mode=_lib.FL_MODE_F64)
        assert abs(info["iterations"] - its_p) <= 3, (alpha, info)


def test_full_size_3d_256_backward_euler_step():
    """256^3, alpha = 1.5, dt = 1e-3, u0 = 16 Gaussians (widths U(0.05, 0.15)),
    f = 0: one mixed-precision backward-Euler step to 1e-8; the residual
    u + dt M u - u0 is checked at sampled points by direct summation."""
    n = 256
    h = 1.0 / (n + 1)
    dt = 1e-3
    u0 = inputs.gaussian_mixture(n, 3, 16, 3, 0.05, 0.15)
    p = Plan(3, (n, n, n), h, 1.5)
    u1, info = p.time_step(gpu(u0), dt, 1.0, tol=1e-8, mode=_lib.FL_MODE_MIXED)
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    u1 = host(u1)
    op = OPlan(3, n, h, 1.5)
    rng = np.random.default_rng(17)
    idx = [tuple(rng.integers(0, n, 3)) for _ in range(4)] + [(128, 128, 128), (5, 250, 131)]
    mu = _direct_samples(op, u1, idx)
    res = np.array([u1[i] + dt * m - u0[i] for i, m in zip(idx, mu)])
    assert np.max(np.abs(res)) <= 1e-7 * np.abs(u0).max()
