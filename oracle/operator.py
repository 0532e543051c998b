"""The discrete fractional Laplacian M of eq. linearelliptic (paper Sec. 3.1).

    (M u)_i = C h^d [ A_{1,d} u_i - sum_{j in J, j != i} u_j / |y_i - y_j|^{d+alpha}
                      + (A_{2,d} + A_{3,d}) L_FD u_i ],

with L_FD u_i = h^{-2} (sum_{|i-j|_1 = 1} u_j - 2d u_i) (Sec. 2.6; reading:
the printed "2^d" is read as 2d, the diagonal of the standard stencil) and
u = 0 outside Omega (extended Dirichlet condition, eq. fracelliptic).

Two evaluations of the same matrix:

* ``dense_matrix`` / ``apply_direct``: the definition summed term by term
  (O(N^2)); for small grids.
* ``apply_fft``: M is block Toeplitz with Toeplitz blocks, so y = M u is a
  linear convolution of the zero-extended u with the kernel k(m) on offsets
  |m_i| <= n_i - 1, computed with a circular embedding of length
  L_i >= 2 n_i - 1 and scipy's FFT (Sec. 3.1, "Forward operator and
  application with FFT").  Any such L gives the identical result.

Grids are boxes of n_1 x ... x n_d interior points, row-major (last axis
fastest).  An optional boolean ``mask`` of that shape selects Omega inside
the box (occluded Cartesian grids, Sec. 1.1); points outside are ignored on
input and returned as 0.

Test infrastructure only (see the package docstring).
"""

import numpy as np
import scipy.fft

from . import constants as cst


class Plan:
    """Constants and geometry of one discrete operator.

    d: dimension; n: interior points per axis (int or tuple); h: spacing;
    alpha in (0, 2); delta: window radius (default 20 h, the paper's choice
    of "a radius of 20 discretization points", Sec. 4.1); mask: optional
    boolean array of shape n selecting Omega.
    """

    def __init__(self, d, n, h, alpha, delta=None, mask=None):
        self.d = int(d)
        self.n = tuple(int(v) for v in np.broadcast_to(np.asarray(n), (self.d,)))
        self.h = float(h)
        self.alpha = float(alpha)
        self.delta = 20.0 * self.h if delta is None else float(delta)
        self.mask = None if mask is None else np.asarray(mask, dtype=bool)
        k = cst.constants(self.d, self.alpha, self.h, self.delta)
        self.C, self.A1, self.A2, self.A3 = k["C"], k["A1"], k["A2"], k["A3"]
        self._khat = None

    # -- entries of M ------------------------------------------------------
    def entry(self, offset):
        """M_{ij} for lattice offset j - i (integer array (..., d))."""
        off = np.asarray(offset, dtype=np.float64)
        dist = np.sqrt(np.sum((off * self.h) ** 2, axis=-1))
        l1 = np.sum(np.abs(off), axis=-1)
        a23 = self.A2 + self.A3
        with np.errstate(divide="ignore"):
            far = -dist ** (-(self.d + self.alpha))
        val = np.where(l1 == 0, self.A1 - 2 * self.d * a23 / self.h ** 2,
                       far + np.where(l1 == 1, a23 / self.h ** 2, 0.0))
        return self.C * self.h ** self.d * val

    def points(self):
        """Integer grid indices of the points of Omega, shape (N, d)."""
        grids = np.meshgrid(*[np.arange(v) for v in self.n], indexing="ij")
        idx = np.stack([g.ravel() for g in grids], axis=1)
        if self.mask is not None:
            idx = idx[self.mask.ravel()]
        return idx

    # -- direct summation ----------------------------------------------------
    def dense_matrix(self):
        """M restricted to Omega as a dense (N, N) array (row-major order of
        the points of Omega)."""
        p = self.points()
        return self.entry(p[None, :, :] - p[:, None, :])

    def apply_direct(self, u):
        """y = M u by direct summation; u, y have the box shape n."""
        u = np.asarray(u, dtype=np.float64).reshape(self.n)
        p = self.points()
        vals = u[tuple(p.T)]
        y = np.zeros(self.n)
        y[tuple(p.T)] = self.dense_matrix() @ vals
        return y

    # -- FFT apply ---------------------------------------------------------
    def fft_shape(self):
        """Circular-embedding lengths: the smallest even L_i >= 2 n_i - 1."""
        return tuple(2 * v for v in self.n)

    def kernel_hat(self):
        """FFT of the kernel k(m), |m_i| <= n_i - 1, embedded circularly."""
        if self._khat is None:
            shape = self.fft_shape()
            axes = []
            for ni, li in zip(self.n, shape):
                m = np.arange(li)
                m = np.where(m <= li // 2, m, m - li)
                axes.append(m)
            grids = np.meshgrid(*axes, indexing="ij")
            off = np.stack(grids, axis=-1)
            k = self.entry(off)
            for ax, ni in enumerate(self.n):
                outside = np.abs(off[..., ax]) > ni - 1
                k = np.where(outside, 0.0, k)
            self._khat = scipy.fft.fftn(k)
        return self._khat

    def apply_fft(self, u, workers=None):
        """y = M u by zero-padded FFT convolution, restricted to Omega."""
        u = np.asarray(u, dtype=np.float64).reshape(self.n)
        if self.mask is not None:
            u = np.where(self.mask, u, 0.0)
        shape = self.fft_shape()
        uh = scipy.fft.fftn(u, s=shape, workers=workers)
        y = scipy.fft.ifftn(uh * self.kernel_hat(), workers=workers)
        y = np.real(y[tuple(slice(0, v) for v in self.n)])
        if self.mask is not None:
            y = np.where(self.mask, y, 0.0)
        return np.ascontiguousarray(y)

    apply = apply_fft
