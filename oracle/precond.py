"""The finite-difference part of the split M = C h^d (K + L) (paper Sec. 3.1,
"Preconditioning: Laplacian pattern and fast Poisson solver").

    L_ij = (A2 + A3)/h^2        for |i - j|_1 = 1,
    L_ii = -2d (A2 + A3)/h^2    (reading: "2^d" printed, 2d meant),

which, since A2 + A3 < 0, is a positive multiple of the standard Dirichlet
finite-difference negative Laplacian.  The preconditioner of the elliptic
solve is P = C h^d L; that of a time step is P = I + theta dt C h^d L
(Sec. 3.2, with theta = 1/2 for Crank-Nicolson).

On a box, L is diagonalised by the type-I discrete sine transform along each
axis (a "fast Poisson solver", Sec. 3.1).  ``solve_box`` uses scipy's
orthonormal DST-I as a library step: z = S diag(1/(shift + scale*lam)) S r.

Test infrastructure only (see the package docstring).
"""

import numpy as np
import scipy.fft
import scipy.sparse as sps


def fd_matrix(plan):
    """C h^d L restricted to the points of Omega, as a sparse (N, N) matrix."""
    p = plan.points()
    index = {tuple(q): i for i, q in enumerate(p)}
    a23 = plan.A2 + plan.A3
    scale = plan.C * plan.h ** plan.d * a23 / plan.h ** 2
    rows, cols, vals = [], [], []
    for i, q in enumerate(p):
        rows.append(i)
        cols.append(i)
        vals.append(-2 * plan.d * scale)
        for ax in range(plan.d):
            for s in (-1, 1):
                nb = list(q)
                nb[ax] += s
                j = index.get(tuple(nb))
                if j is not None:
                    rows.append(i)
                    cols.append(j)
                    vals.append(scale)
    n = len(p)
    return sps.csr_matrix((vals, (rows, cols)), shape=(n, n))


def eigenvalues(plan):
    """Eigenvalues of C h^d L on the full box, indexed like the DST-I output:
    lambda_k = C h^d (A2+A3)/h^2 * sum_i (2 cos(pi k_i/(n_i+1)) - 2),
    k_i = 1..n_i."""
    a23 = plan.A2 + plan.A3
    scale = plan.C * plan.h ** plan.d * a23 / plan.h ** 2
    lam = np.zeros(plan.n)
    for ax, ni in enumerate(plan.n):
        k = np.arange(1, ni + 1)
        e = 2.0 * np.cos(np.pi * k / (ni + 1)) - 2.0
        shape = [1] * plan.d
        shape[ax] = ni
        lam = lam + e.reshape(shape)
    return scale * lam


def _dst_solve(plan, r, shift, scale):
    r = np.asarray(r, dtype=np.float64).reshape(plan.n)
    rh = scipy.fft.dstn(r, type=1, norm="ortho")
    zh = rh / (shift + scale * eigenvalues(plan))
    return scipy.fft.idstn(zh, type=1, norm="ortho")


def solve_box(plan, r, shift=0.0, scale=1.0):
    """z = (shift I + scale C h^d L)^{-1} r on the full box by DST-I."""
    if plan.mask is not None and not plan.mask.all():
        raise ValueError("the DST preconditioner needs a full box")
    return _dst_solve(plan, r, shift, scale)


def solve_embedded(plan, r, shift=0.0, scale=1.0):
    """A cheaper preconditioner of an occluded domain Omega inside the box
    (not the paper's choice, which is L on Omega itself, solve_domain): z = R (shift I + scale C h^d L_box)^{-1} R^T r with R the
    restriction to Omega, i.e. zero the residual outside Omega, solve on the
    box by DST-I, zero the result outside Omega.  R B^{-1} R^T is symmetric
    positive definite on the functions supported in Omega, so CG keeps its
    guarantees.  Equal to solve_box on the full box."""
    r = np.asarray(r, dtype=np.float64).reshape(plan.n)
    m = np.ones(plan.n, bool) if plan.mask is None else plan.mask
    return np.where(m, _dst_solve(plan, np.where(m, r, 0.0), shift, scale), 0.0)


def solve_domain(plan, r, shift=0.0, scale=1.0):
    """The paper's preconditioner on an occluded domain Omega (Sec. 4.4):
    z = (shift I + scale C h^d L_Omega)^{-1} r with L_Omega the
    finite-difference Laplacian on the points of Omega and Dirichlet
    conditions on every point outside it (fd_matrix keeps only neighbours in
    Omega).  The paper factorises it by sparse Cholesky; here a sparse direct
    solve (scipy's SuperLU) is the library step.  z = 0 outside Omega; equal
    to solve_box on the full box."""
    import scipy.sparse.linalg as spla
    r = np.asarray(r, dtype=np.float64).reshape(plan.n)
    m = np.ones(plan.n, bool) if plan.mask is None else plan.mask
    A = (scale * fd_matrix(plan) + shift * sps.identity(int(m.sum()))).tocsc()
    z = np.zeros(plan.n)
    z[m] = spla.spsolve(A, r[m])
    return z


# -- other members of the family (shift I + scale C h^d L) ---------------------
#
# Every preconditioner below is P = pshift I + pscale C h^d L on the box
# (restricted to Omega as in solve_embedded), for the operator
# sigma I + tau M (sigma = 0, tau = 1: the elliptic problem; sigma = 1,
# tau = theta dt: a time step).  The paper's choice is pshift = sigma,
# pscale = tau.


def stencil_params(plan, sigma=0.0, tau=1.0):
    """The alternative the paper mentions after its preconditioner (Sec. 3.1):
    M~ = M with every entry outside the (2d+1)-point stencil set to zero.
    By the entries of M,

        M~ = C h^d [A1 I - h^-(d+alpha) S] + C h^d L,

    S the nearest-neighbour sum.  With g = C h^d (A2+A3)/h^2 (< 0) and
    C h^d L = g (S - 2d I) this is pshift I + pscale C h^d L with
    pscale = 1 + C h^-alpha / |g| and pshift = C h^d (A1 - 2d h^-(d+alpha)).
    Returns (pshift, pscale) of sigma I + tau M~."""
    g = plan.C * plan.h ** plan.d * (plan.A2 + plan.A3) / plan.h ** 2
    kappa = plan.C * plan.h ** (-plan.alpha)
    ps = plan.C * plan.h ** plan.d * (plan.A1 - 2 * plan.d * plan.h ** (-(plan.d + plan.alpha)))
    return sigma + tau * ps, tau * (1.0 + kappa / abs(g))


def sine_mode(n, k):
    """The separable DST-I eigenvector of L with wave numbers k (one per
    axis): v_i = prod_a sin(pi k_a (i_a + 1) / (n_a + 1)), i_a = 0..n_a-1."""
    v = np.ones(n)
    for ax, (ni, ki) in enumerate(zip(n, k)):
        s = np.sin(np.pi * ki * np.arange(1, ni + 1) / (ni + 1))
        shape = [1] * len(n)
        shape[ax] = ni
        v = v * s.reshape(shape)
    return v


def extreme_quotients(plan, apply=None):
    """Rayleigh quotients of the operator (default plan.apply) on the
    lowest (k = 1 on every axis) and highest (k = n) sine modes, restricted
    to Omega, and the eigenvalues of C h^d L on the box for those modes.
    Returns (mu_lo, mu_hi, lam_lo, lam_hi)."""
    apply = plan.apply if apply is None else apply
    m = np.ones(plan.n, bool) if plan.mask is None else plan.mask
    lam = eigenvalues(plan)
    out = []
    for k in ((1,) * plan.d, plan.n):
        v = np.where(m, sine_mode(plan.n, k), 0.0)
        out.append(float(np.sum(v * apply(v)) / np.sum(v * v)))
    return out[0], out[1], float(lam.flat[0]), float(lam.flat[-1])


def balanced_params(plan, sigma=0.0, tau=1.0, apply=None):
    """FD preconditioner with a shift (not in the paper): P = x I + tau C h^d L
    with x chosen so that the preconditioned operator's ratio
    (sigma + tau mu) / (x + tau lam) is the same on the lowest and highest
    sine modes:

        x = tau (A lam_hi - B lam_lo) / (B - A),
        A = sigma + tau mu_lo,  B = sigma + tau mu_hi,

    kept >= 0 (P stays positive definite).  The symbol of M grows like
    |xi|^alpha and that of L like |xi|^2; the shift flattens their ratio at
    low frequencies, which the paper's choice (x = sigma) leaves growing like
    |xi|^(alpha-2).  For a time step with a small tau the balance can lie
    below sigma.
    Returns (pshift, pscale) = (x, tau)."""
    mu_lo, mu_hi, lam_lo, lam_hi = extreme_quotients(plan, apply)
    a = sigma + tau * mu_lo
    b = sigma + tau * mu_hi
    x = tau * (a * lam_hi - b * lam_lo) / (b - a) if b > a else sigma
    return max(0.0, x), tau
