"""Solvers of paper Sec. 3: CG / PCG for M u = f (Sec. 3.1), the implicit
theta time step (eq. timestepping, Sec. 3.2; theta = 1/2 is the paper's
Crank-Nicolson, theta = 1 backward Euler), and FP32-inner / FP64-outer
iterative refinement.

Readings (the paper is silent on these details):

* stopping rule: ||r_k||_2 <= tol * ||b||_2 with the recursive residual r_k,
  x_0 = 0 for the elliptic problem and x_0 = u^(k) for a time step
  (warm start, Sec. 4.5); the iteration count is the number of operator
  applications inside the loop;
* iteration caps of 1000 (1D/2D) and 250 (3D) are the paper's (Sec. 4);
* refinement: r = f - M u in FP64, the correction solves M d = r with PCG
  run entirely in float32 arrays to a relative tolerance ``inner_tol``, then
  u += d; stop when ||f - M u|| <= tol ||f||.

Test infrastructure only (see the package docstring).
"""

import numpy as np

from . import precond as pc


def pcg(apply_a, b, precond=None, x0=None, tol=1e-9, maxit=1000,
        dtype=np.float64):
    """Preconditioned conjugate gradients (Hestenes-Stiefel).

    apply_a, precond: callables on arrays of b's shape.  Vectors are kept in
    ``dtype``; inner products are accumulated in float64.
    Returns (x, iterations, converged, residual_history)."""
    b = np.asarray(b).astype(dtype)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0).astype(dtype).copy()
    r = b - apply_a(x).astype(dtype) if x0 is not None else b.copy()
    bnorm = np.sqrt(np.sum(b.astype(np.float64) ** 2))
    hist = [np.sqrt(np.sum(r.astype(np.float64) ** 2))]
    if bnorm == 0.0:
        return x, 0, True, hist
    if hist[-1] <= tol * bnorm:
        return x, 0, True, hist
    z = (precond(r) if precond is not None else r).astype(dtype)
    p = z.copy()
    rz = np.sum(r.astype(np.float64) * z)
    for it in range(1, maxit + 1):
        q = apply_a(p).astype(dtype)
        pq = np.sum(p.astype(np.float64) * q)
        alpha = rz / pq
        x = (x + dtype(alpha) * p).astype(dtype)
        r = (r - dtype(alpha) * q).astype(dtype)
        rn = np.sqrt(np.sum(r.astype(np.float64) ** 2))
        hist.append(rn)
        if rn <= tol * bnorm:
            return x, it, True, hist
        z = (precond(r) if precond is not None else r).astype(dtype)
        rz_new = np.sum(r.astype(np.float64) * z)
        beta = rz_new / rz
        rz = rz_new
        p = (z + dtype(beta) * p).astype(dtype)
    return x, maxit, False, hist


def solve_elliptic(plan, f, tol=1e-9, maxit=1000, precondition=True):
    """Solve M u = f (eq. matelliptic) by CG, optionally preconditioned with
    C h^d L applied by the DST fast solver (Sec. 3.1)."""
    prec = (lambda r: pc.solve_box(plan, r)) if precondition else None
    return pcg(plan.apply, f, prec, None, tol, maxit)


def theta_rhs(plan, u_prev, dt, theta, f_prev=None, f_next=None):
    """b = (I - (1-theta) dt M) u^(k) + dt (theta f^(k+1) + (1-theta) f^(k))
    (eq. timestepping with theta = 1/2 generalised to theta in [0, 1])."""
    b = np.asarray(u_prev, dtype=np.float64).copy()
    if theta != 1.0:
        b = b - (1.0 - theta) * dt * plan.apply(u_prev)
    if f_next is not None:
        b = b + dt * theta * np.asarray(f_next, dtype=np.float64)
    if f_prev is not None and theta != 1.0:
        b = b + dt * (1.0 - theta) * np.asarray(f_prev, dtype=np.float64)
    return b


def theta_step(plan, u_prev, dt, theta=1.0, f_prev=None, f_next=None,
               tol=1e-9, maxit=1000, precondition=True, x0="warm"):
    """One implicit step (I + theta dt M) u^(k+1) = b (Sec. 3.2) by PCG with
    preconditioner I + theta dt C h^d L (Sec. 3.2), warm-started from
    u^(k) unless x0 is given (None means a zero initial guess)."""
    b = theta_rhs(plan, u_prev, dt, theta, f_prev, f_next)
    a = lambda v: v + theta * dt * plan.apply(v)
    prec = ((lambda r: pc.solve_box(plan, r, 1.0, theta * dt))
            if precondition else None)
    start = u_prev if isinstance(x0, str) else x0
    return pcg(a, b, prec, start, tol, maxit)


def refine_mixed(plan, f, tol=1e-8, inner_tol=1e-4, max_outer=30,
                 inner_maxit=1000, shift=0.0, scale=1.0, u0=None):
    """FP64 iterative refinement around a float32 PCG for
    (shift I + scale M) u = f with preconditioner shift I + scale C h^d L.
    shift = 0, scale = 1 is the elliptic problem; shift = 1,
    scale = theta dt a time step.  Returns (u, outer, inner_total, relres)."""
    f = np.asarray(f, dtype=np.float64)
    u = np.zeros_like(f) if u0 is None else np.asarray(u0, np.float64).copy()
    fnorm = np.linalg.norm(f)
    op64 = lambda v: shift * v + scale * plan.apply(v)

    def op32(v):
        return (shift * v.astype(np.float64)
                + scale * plan.apply(v.astype(np.float64))).astype(np.float32)

    def pre32(r):
        z = pc.solve_box(plan, r.astype(np.float64), shift if shift else 0.0,
                         scale)
        return z.astype(np.float32)

    inner_total = 0
    for outer in range(max_outer + 1):
        r = f - op64(u)
        rel = np.linalg.norm(r) / fnorm if fnorm > 0 else 0.0
        if rel <= tol:
            return u, outer, inner_total, rel
        if outer == max_outer:
            break
        d, its, _, _ = pcg(op32, r.astype(np.float32), pre32, None, inner_tol,
                           inner_maxit, dtype=np.float32)
        inner_total += its
        u = u + d.astype(np.float64)
    return u, max_outer, inner_total, rel
