"""Pins for the shifted members of the preconditioner family in
oracle/precond.py: the stencil part M~ of M (the alternative the paper
mentions after its preconditioner, Sec. 3.1) and the balanced shift (not
in the paper).  Each is checked against the dense matrix of M summed term by
term, against a closed form, or by its effect on CG."""

import numpy as np
import pytest

from oracle import precond as pc
from oracle import solvers
from oracle.operator import Plan


def _stencil_of(A, pts):
    """A with every entry outside the (2d+1)-point stencil set to zero."""
    l1 = np.abs(pts[None, :, :] - pts[:, None, :]).sum(axis=-1)
    return np.where(l1 <= 1, A, 0.0)


@pytest.mark.parametrize("d,n,alpha,sigma,tau", [
    (2, (7, 6), 1.3, 0.0, 1.0),
    (2, (5, 9), 0.6, 1.0, 0.02),
    (3, (4, 5, 3), 1.7, 0.0, 1.0),
    (3, (3, 4, 4), 0.9, 1.0, 0.5),
])
def test_stencil_params_are_M_on_its_stencil(d, n, alpha, sigma, tau):
    """sigma I + tau M~ built from (pshift, pscale) equals the dense matrix
    of sigma I + tau M with the entries off the stencil zeroed."""
    p = Plan(d, n, 1.0 / (max(n) + 1), alpha)
    pts = p.points()
    A = sigma * np.eye(len(pts)) + tau * p.dense_matrix()
    want = _stencil_of(A, pts)
    ps, sc = pc.stencil_params(p, sigma, tau)
    got = ps * np.eye(len(pts)) + sc * pc.fd_matrix(p).toarray()
    assert np.allclose(got, want, rtol=0, atol=1e-12 * abs(want).max())
    # positive definite, as the paper's remark needs
    assert np.linalg.eigvalsh(got).min() > 0


@pytest.mark.parametrize("d,n", [(2, (6, 9)), (3, (4, 3, 5))])
def test_sine_modes_are_the_extreme_eigenvectors_of_L(d, n):
    p = Plan(d, n, 0.1, 1.2)
    L = pc.fd_matrix(p).toarray()
    lam = pc.eigenvalues(p)
    for k, want in (((1,) * d, lam.flat[0]), (n, lam.flat[-1])):
        v = pc.sine_mode(n, k).ravel()
        assert np.allclose(L @ v, want * v, rtol=0, atol=1e-12 * abs(want))
    assert lam.flat[0] == lam.min() and lam.flat[-1] == lam.max()


@pytest.mark.parametrize("sigma,tau,a", [(0.0, 1.0, 3.7), (1.0, 0.05, 20.0), (0.5, 2.0, 0.0)])
def test_balanced_shift_recovers_a_shifted_laplacian(sigma, tau, a):
    """When the operator is itself a I + C h^d L, the balanced preconditioner
    is that operator exactly: pshift = sigma + tau a, and CG converges in
    one step."""
    p = Plan(2, (11, 8), 1.0 / 12, 1.1)
    F = pc.fd_matrix(p)
    op = lambda v: a * v + (F @ v.ravel()).reshape(v.shape)
    ps, sc = pc.balanced_params(p, sigma, tau, apply=op)
    assert sc == tau
    assert ps == pytest.approx(sigma + tau * a, rel=1e-10, abs=1e-12)
    b = np.random.default_rng(3).standard_normal(p.n)
    A = lambda v: sigma * v + tau * op(v)
    _, its, ok, _ = solvers.pcg(A, b, lambda r: pc.solve_box(p, r, ps, sc), tol=1e-10)
    assert ok and its == 1


@pytest.mark.parametrize("alpha", [0.7, 1.5])
def test_balanced_ratio_is_equal_on_the_extreme_modes(alpha):
    """The defining property, checked with the dense matrix of M (not the
    FFT apply the function uses)."""
    p = Plan(2, (9, 10), 1.0 / 11, alpha)
    M = p.dense_matrix()
    F = pc.fd_matrix(p).toarray()
    for sigma, tau in ((0.0, 1.0), (1.0, 0.1)):
        x, sc = pc.balanced_params(p, sigma, tau)
        ratios = []
        for k in ((1, 1), p.n):
            v = pc.sine_mode(p.n, k).ravel()
            num = v @ (sigma * v + tau * (M @ v))
            den = v @ (x * v + sc * (F @ v))
            ratios.append(num / den)
        assert ratios[0] == pytest.approx(ratios[1], rel=1e-10)


def test_masked_quotients_use_modes_restricted_to_omega():
    mask = np.ones((12, 12), bool)
    mask[6:, 6:] = False
    p = Plan(2, mask.shape, 1.0 / 13, 1.25, mask=mask)
    M = p.dense_matrix()
    idx = np.flatnonzero(mask.ravel())
    mu_lo, mu_hi, _, _ = pc.extreme_quotients(p)
    for k, mu in (((1, 1), mu_lo), (p.n, mu_hi)):
        v = pc.sine_mode(p.n, k).ravel()[idx]
        assert mu == pytest.approx(v @ M @ v / (v @ v), rel=1e-11)


def test_shifted_preconditioners_against_the_paper_choice():
    """At alpha = 1 the balanced shift needs far fewer CG iterations than L
    alone and than plain CG; at alpha = 1.75 the stencil part M~ is worse
    than L (the paper found no benefit in it).  All reach the dense-LU
    solution."""
    n = 31
    rng = np.random.default_rng(11)
    for alpha in (1.0, 1.75):
        p = Plan(2, n, 1.0 / (n + 1), alpha)
        f = rng.standard_normal(p.n)
        u_lu = np.linalg.solve(p.dense_matrix(), f.ravel()).reshape(p.n)
        its = {}
        for name, prm in (("L", (0.0, 1.0)), ("stencil", pc.stencil_params(p)),
                          ("balanced", pc.balanced_params(p))):
            u, k, ok, _ = solvers.pcg(p.apply, f, lambda r: pc.solve_box(p, r, *prm), tol=1e-11)
            assert ok
            assert np.abs(u - u_lu).max() <= 1e-8 * np.abs(u_lu).max()
            its[name] = k
        its["plain"] = solvers.pcg(p.apply, f, None, tol=1e-11, maxit=2000)[1]
        if alpha == 1.0:
            assert its["balanced"] < 0.6 * its["L"] and its["balanced"] < 0.6 * its["plain"]
        else:
            assert its["stencil"] > its["L"] and its["balanced"] <= its["L"]


# -- the paper's preconditioner on occluded domains (Sec. 4.4) -----------------

def _l_shape(n):
    m = n - 1
    mask = np.ones((m, m), dtype=bool)
    mask[m - n // 2:, m - n // 2:] = False
    return mask


def _octagon(n):
    i = np.arange(1, n)
    a = np.minimum(i, n - i)
    return (a[:, None] + a[None, :]) > n // 4


def test_solve_domain_is_the_box_solve_on_the_full_box():
    p = Plan(2, (9, 12), 0.05, 1.3)
    r = np.random.default_rng(40).standard_normal((9, 12))
    for shift, scale in ((0.0, 1.0), (1.0, 0.3)):
        assert np.allclose(pc.solve_domain(p, r, shift, scale), pc.solve_box(p, r, shift, scale),
                           rtol=0, atol=1e-12 * np.abs(pc.solve_box(p, r, shift, scale)).max())


def test_solve_domain_has_dirichlet_conditions_on_the_hole():
    """z solves the shifted FD equation at every point of Omega with z = 0
    at the hole's points (the 5-point stencil written out here)."""
    n = 16
    mask = _l_shape(n)
    p = Plan(2, mask.shape, 1.0 / n, 1.6, mask=mask)
    r = np.where(mask, np.random.default_rng(41).standard_normal(mask.shape), 0.0)
    shift, scale = 0.7, 1.3
    z = pc.solve_domain(p, r, shift, scale)
    assert np.all(z[~mask] == 0.0)
    g = p.C * p.h ** 2 * (p.A2 + p.A3) / p.h ** 2       # C h^d L = g (S - 4 I), g < 0
    zp = np.pad(z, 1)
    s = zp[:-2, 1:-1] + zp[2:, 1:-1] + zp[1:-1, :-2] + zp[1:-1, 2:]
    lhs = shift * z + scale * g * (s - 4 * z)
    assert np.allclose(lhs[mask], r[mask], rtol=0, atol=1e-10 * np.abs(r).max())


@pytest.mark.parametrize("shape,paper", [("lshape", (10, 14)), ("octagon", (10, 14))])
def test_occluded_iteration_counts_of_the_paper(shape, paper):
    """Tables tab:L2 and tab:octagon2, first row (n = 128: N = 12033 and
    14145), alpha = 1.75, f = 1 on Omega, CG with L_Omega: the printed
    preconditioned counts at 1e-6 and 1e-9."""
    n = 128
    mask = _l_shape(n) if shape == "lshape" else _octagon(n)
    assert int(mask.sum()) == (12033 if shape == "lshape" else 14145)
    p = Plan(2, mask.shape, 1.0 / n, 1.75, mask=mask)
    f = np.where(mask, 1.0, 0.0)
    its = tuple(solvers.pcg(p.apply, f, lambda r: pc.solve_domain(p, r), None, tol, 1000)[1]
                for tol in (1e-6, 1e-9))
    assert its == paper
