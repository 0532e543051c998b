"""Constants of the quadrature (paper Sec. 2.5-2.7).  FP64, plain NumPy/SciPy.

All quantities are in the paper's physical units: lattice spacing h,
window radius delta, lattice points y_j = j h.

* ``c_alpha_d``      -- the normalising constant C_{alpha,d} of eq. fl.
  The paper does not print it (it cites its "known" value); we use the
  standard value 2^alpha Gamma((d+alpha)/2) / (pi^{d/2} |Gamma(-alpha/2)|).
* ``window``         -- W_delta of eq. window.
* ``lattice_zeta``   -- Z_d(alpha) = sum_{m in Z^d, m != 0} |m|^{-(d+alpha)},
  so that A_{1,d} = h^{-(d+alpha)} Z_d (eq. int1constants).  The paper
  evaluates this lattice sum by Chebyshev far-field compression (end of
  Sec. 2.7); we evaluate the same number by the Ewald / theta-function
  split, which converges exponentially.
* ``a1``, ``a2``, ``a3`` -- A_{1,d}, A_{2,d} (eq. int1constants) and
  A_{3,d} (eq. a3).  A_{3,d} uses the closed form available for the
  polynomial window (Sec. 2.7).

Test infrastructure only (see the package docstring).
"""

import math

import numpy as np
from scipy import special


def c_alpha_d(alpha, d):
    """C_{alpha,d} of eq. fl (reading: the standard normalisation)."""
    return (2.0 ** alpha * math.gamma((d + alpha) / 2.0)
            / (math.pi ** (d / 2.0) * abs(math.gamma(-alpha / 2.0))))


def window(r, delta):
    """W_delta(r) of eq. window: 1 - 35 t^4 + 84 t^5 - 70 t^6 + 20 t^7 for
    t = r/delta < 1, zero otherwise."""
    t = np.asarray(r, dtype=np.float64) / delta
    p = 1.0 - 35.0 * t**4 + 84.0 * t**5 - 70.0 * t**6 + 20.0 * t**7
    return np.where(t < 1.0, p, 0.0)


def _upper_gamma(a, x):
    """Non-normalised upper incomplete gamma Gamma(a, x) for x > 0 and any
    real a > -1 (a != 0).  For a <= 0 it uses Gamma(a, x) =
    (Gamma(a+1, x) - x^a e^{-x}) / a."""
    x = np.asarray(x, dtype=np.float64)
    if a > 0:
        return special.gammaincc(a, x) * special.gamma(a)
    return (special.gammaincc(a + 1.0, x) * special.gamma(a + 1.0)
            - x ** a * np.exp(-x)) / a


def _lattice(d, radius):
    """All integer points m in [-radius, radius]^d except 0, shape (K, d)."""
    ax = np.arange(-radius, radius + 1)
    grids = np.meshgrid(*([ax] * d), indexing="ij")
    m = np.stack([g.ravel() for g in grids], axis=1).astype(np.float64)
    return m[np.any(m != 0, axis=1)]


def lattice_zeta(d, alpha, radius=8):
    """Z_d(alpha) = sum_{m != 0} |m|^{-s}, s = d + alpha, by the Ewald split

        pi^{-s/2} Gamma(s/2) Z = sum_{m != 0} [ (pi|m|^2)^{-s/2} Gamma(s/2, pi|m|^2)
                                 + (pi|m|^2)^{(s-d)/2} Gamma((d-s)/2, pi|m|^2) ]
                                 + 2/(s-d) - 2/s,

    obtained from |m|^{-s} = pi^{s/2}/Gamma(s/2) int_0^inf t^{s/2-1}
    e^{-pi t |m|^2} dt, splitting at t = 1 and using the theta-function
    identity theta(t) = t^{-d/2} theta(1/t).  Terms decay like
    e^{-pi |m|^2}; radius 8 leaves < 1e-80 relative truncation."""
    s = d + alpha
    m = _lattice(d, radius)
    x = math.pi * np.sum(m * m, axis=1)
    terms = (x ** (-s / 2.0) * _upper_gamma(s / 2.0, x)
             + x ** ((s - d) / 2.0) * _upper_gamma((d - s) / 2.0, x))
    total = np.sum(terms) + 2.0 / (s - d) - 2.0 / s
    return total * math.pi ** (s / 2.0) / math.gamma(s / 2.0)


def a1(d, alpha, h):
    """A_{1,d} of eq. int1constants: sum over the whole lattice hZ^d minus
    the origin of |y_j|^{-(d+alpha)} (reading: infinite lattice, not the
    truncated domain)."""
    return h ** (-(d + alpha)) * lattice_zeta(d, alpha)


def a2(d, alpha, h, delta):
    """A_{2,d} of eq. int1constants: (1/2) sum_{j != 0} W_delta(|y_j|)
    (e_1^T y_j)^2 / |y_j|^{d+alpha}; only |y_j| < delta contribute."""
    radius = int(math.ceil(delta / h)) + 1
    y = _lattice(d, radius) * h
    r = np.sqrt(np.sum(y * y, axis=1))
    return 0.5 * np.sum(window(r, delta) * y[:, 0] ** 2 / r ** (d + alpha))


def sphere_area(d):
    """|S^{d-1}|, the surface area of the unit sphere in R^d (2 for d=1)."""
    return 2.0 * math.pi ** (d / 2.0) / math.gamma(d / 2.0)


def window_moment(alpha):
    """P(alpha) = int_0^1 W_1(t) t^{1-alpha} dt for the polynomial window of
    eq. window, integrated term by term."""
    return (1.0 / (2.0 - alpha) - 35.0 / (6.0 - alpha) + 84.0 / (7.0 - alpha)
            - 70.0 / (8.0 - alpha) + 20.0 / (9.0 - alpha))


def a3(d, alpha, h, delta):
    """A_{3,d} of eq. a3: -(h^{-d}/2) int_{R^d} W_delta(|y|) (e_1^T y)^2 /
    |y|^{d+alpha} dy.  In polar coordinates the angular mean of (e_1^T y)^2
    is r^2/d, so the integral is (|S^{d-1}|/d) delta^{2-alpha} P(alpha)."""
    integral = sphere_area(d) / d * delta ** (2.0 - alpha) * window_moment(alpha)
    return -0.5 * h ** (-d) * integral


def constants(d, alpha, h, delta):
    """Dict with C = C_{alpha,d}, A1, A2, A3 for one plan."""
    return {
        "C": c_alpha_d(alpha, d),
        "A1": a1(d, alpha, h),
        "A2": a2(d, alpha, h, delta),
        "A3": a3(d, alpha, h, delta),
    }
