"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the solver's arithmetic: it only draws random
numbers and samples Gaussian mixtures / the paper's test functions on the
interior grid of the unit box.

Grid convention: Omega = [0, 1]^d with n interior points per axis at
x_j = j h, j = 1..n, h = 1/(n+1); arrays are row-major with the last axis
fastest.

Gaussian mixture (the stand-in for the paper's smooth synthetic data):
    g(x) = sum_b a_b exp(-|x - c_b|^2 / (2 w_b^2)),
with, per bump and in this draw order from numpy's PCG64 generator seeded
with ``seed``: the centre c_b (d uniforms on [0, 1)), the width
w_b ~ U(w_lo, w_hi), the amplitude a_b ~ N(0, 1).
"""

import numpy as np


def grid_axes(n, d):
    """Coordinates x_j = j/(n+1), j = 1..n, for each of the d axes."""
    n = np.broadcast_to(np.asarray(n), (d,))
    return [np.arange(1, int(v) + 1, dtype=np.float64) / (int(v) + 1.0) for v in n]


def gaussian_params(d, bumps, seed, w_lo, w_hi):
    """Centres (bumps, d), widths (bumps,), amplitudes (bumps,)."""
    rng = np.random.default_rng(seed)
    c = np.empty((bumps, d))
    w = np.empty(bumps)
    a = np.empty(bumps)
    for b in range(bumps):
        c[b] = rng.random(d)
        w[b] = rng.uniform(w_lo, w_hi)
        a[b] = rng.standard_normal()
    return c, w, a


def gaussian_mixture(n, d, bumps, seed, w_lo=0.05, w_hi=0.2, dtype=np.float64):
    """Sum of ``bumps`` seeded Gaussians sampled at the interior grid points."""
    axes = grid_axes(n, d)
    shape = tuple(len(x) for x in axes)
    c, w, a = gaussian_params(d, bumps, seed, w_lo, w_hi)
    out = np.zeros(shape)
    for b in range(bumps):
        # separable: exp(-|x-c|^2/(2w^2)) = prod_i exp(-(x_i-c_i)^2/(2w^2))
        term = np.array(a[b])
        for i, x in enumerate(axes):
            g = np.exp(-((x - c[b, i]) ** 2) / (2.0 * w[b] ** 2))
            sh = [1] * d
            sh[i] = len(x)
            term = term * g.reshape(sh)
        out = out + term
    return out.astype(dtype)


def random_field(n, d, seed, dtype=np.float64):
    """Standard normal values at the interior grid points (the paper's
    "random RHS" of the single-time-step experiment, Sec. 4.5)."""
    shape = tuple(int(v) for v in np.broadcast_to(np.asarray(n), (d,)))
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def cosine_product(n, d, nu=(3, 11, 2)):
    """u0(x) = prod_i (1/4)(1 + cos(2 pi nu_i x_i - pi))^2, the initial
    condition of the paper's time-dependent example (Sec. 4.5); nu = 1 in
    every axis gives the function g_1 of eq. test."""
    axes = grid_axes(n, d)
    out = np.array(1.0)
    for i, x in enumerate(axes):
        g = 0.25 * (1.0 + np.cos(2.0 * np.pi * nu[i] * x - np.pi)) ** 2
        sh = [1] * d
        sh[i] = len(x)
        out = out * g.reshape(sh)
    return out


def alpha_draws(count, seed, lo=0.3, hi=1.8):
    """alpha ~ U(lo, hi) per problem, seeded."""
    return np.random.default_rng(seed).uniform(lo, hi, size=count)


def batch_sides(count, seed, sides=tuple(range(96, 769, 32))):
    """Grid sides drawn uniformly from ``sides`` (default 96, 128, ..., 768)."""
    rng = np.random.default_rng(seed)
    return [int(sides[i]) for i in rng.integers(0, len(sides), size=count)]
