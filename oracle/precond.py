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
    """Preconditioner of an occluded domain Omega inside the box (not the
    paper's choice, which is a sparse Cholesky factorisation of L on Omega,
    Sec. 4.4): z = R (shift I + scale C h^d L_box)^{-1} R^T r with R the
    restriction to Omega, i.e. zero the residual outside Omega, solve on the
    box by DST-I, zero the result outside Omega.  R B^{-1} R^T is symmetric
    positive definite on the functions supported in Omega, so CG keeps its
    guarantees.  Equal to solve_box on the full box."""
    r = np.asarray(r, dtype=np.float64).reshape(plan.n)
    m = np.ones(plan.n, bool) if plan.mask is None else plan.mask
    return np.where(m, _dst_solve(plan, np.where(m, r, 0.0), shift, scale), 0.0)
