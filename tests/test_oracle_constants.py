"""Pins for oracle/constants.py against values the paper and mathematics fix
(closed forms of lattice sums, quadrature of the defining integrals)."""

import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import constants as cst


@pytest.mark.parametrize("alpha,d,expected", [
    (1.0, 1, 1.0 / math.pi),          # (-Delta)^{1/2} in 1D: C = 1/pi
    (1.0, 3, 1.0 / math.pi ** 2),     # (-Delta)^{1/2} in 3D: C = 1/pi^2
])
def test_c_alpha_d_special_cases(alpha, d, expected):
    assert cst.c_alpha_d(alpha, d) == pytest.approx(expected, rel=1e-14)


@pytest.mark.parametrize("alpha", [0.3, 0.75, 1.0, 1.5, 1.9])
def test_c_alpha_d_second_form(alpha):
    # alpha 2^{alpha-1} Gamma((d+alpha)/2) / (pi^{d/2} Gamma(1-alpha/2)), the
    # same constant through Gamma(1-alpha/2) = (-alpha/2) Gamma(-alpha/2)
    for d in (1, 2, 3):
        other = (alpha * 2 ** (alpha - 1) * math.gamma((d + alpha) / 2)
                 / (math.pi ** (d / 2) * math.gamma(1 - alpha / 2)))
        assert cst.c_alpha_d(alpha, d) == pytest.approx(other, rel=1e-13)


@pytest.mark.parametrize("alpha", [0.3, 0.75, 1.25, 1.5, 1.9])
def test_lattice_zeta_1d_is_riemann(alpha):
    # Z_1 = 2 zeta(1 + alpha)
    assert cst.lattice_zeta(1, alpha) == pytest.approx(
        2 * special.zeta(1 + alpha), rel=1e-12)


def _dirichlet_beta(t):
    return 4.0 ** (-t) * (special.zeta(t, 0.25) - special.zeta(t, 0.75))


@pytest.mark.parametrize("alpha", [0.3, 0.75, 1.25, 1.5, 1.9])
def test_lattice_zeta_2d_is_zeta_times_beta(alpha):
    # sum over Z^2 of |m|^{-2t} = 4 zeta(t) beta(t), t = (2 + alpha)/2
    t = (2 + alpha) / 2
    assert cst.lattice_zeta(2, alpha) == pytest.approx(
        4 * special.zeta(t) * _dirichlet_beta(t), rel=1e-12)


@pytest.mark.parametrize("alpha", [0.75, 1.5])
def test_lattice_zeta_3d_brute_force(alpha):
    # direct sum over the ball |m| <= R plus the integral of the tail
    s = 3 + alpha
    R = 48
    ax = np.arange(-R, R + 1, dtype=np.float64)
    x, y, z = np.meshgrid(ax, ax, ax, indexing="ij")
    r2 = x * x + y * y + z * z
    sel = (r2 > 0) & (r2 <= R * R)
    part = np.sum(r2[sel] ** (-s / 2))
    tail = 4 * math.pi * R ** (3 - s) / (s - 3)
    assert cst.lattice_zeta(3, alpha) == pytest.approx(part + tail, rel=2e-4)


def test_window_shape():
    delta = 3.0
    r = np.linspace(0, 4, 4001)
    w = cst.window(r, delta)
    assert w[0] == 1.0
    assert np.all(w[r >= delta] == 0.0)
    assert np.all((w >= 0) & (w <= 1))
    assert np.all(np.diff(w[r < delta]) <= 1e-15)       # non-increasing
    # 1 - W = O(t^4) at 0: the window is flat to third order
    t = 1e-3
    assert 1 - cst.window(t * delta, delta) == pytest.approx(35 * t ** 4, rel=1e-2)


@pytest.mark.parametrize("alpha", [0.3, 1.0, 1.75])
def test_window_moment_by_quadrature(alpha):
    val, _ = integrate.quad(lambda t: cst.window(t, 1.0) * t ** (1 - alpha), 0, 1,
                            limit=200)
    assert cst.window_moment(alpha) == pytest.approx(val, rel=1e-9)


@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_a3_2d_by_cartesian_quadrature(alpha):
    # -(h^{-2}/2) * int W(|y|) y1^2 / |y|^{2+alpha} dy, integrand in
    # Cartesian form, integrated over the disk in polar coordinates
    h, delta = 0.1, 2.0

    def f(r, th):
        y1 = r * math.cos(th)
        return cst.window(r, delta) * y1 * y1 / r ** (2 + alpha) * r

    val, _ = integrate.dblquad(f, 0, 2 * math.pi, 0, delta, epsabs=1e-12)
    assert cst.a3(2, alpha, h, delta) == pytest.approx(-0.5 * h ** -2 * val, rel=1e-7)


def test_a3_3d_by_quadrature():
    alpha, h, delta = 1.25, 0.05, 1.0

    def f(r, ph, th):
        y1 = r * math.sin(ph) * math.cos(th)
        return (cst.window(r, delta) * y1 * y1 / r ** (3 + alpha)
                * r * r * math.sin(ph))

    val, _ = integrate.tplquad(f, 0, 2 * math.pi, 0, math.pi, 0, delta,
                               epsabs=1e-10)
    assert cst.a3(3, alpha, h, delta) == pytest.approx(-0.5 * h ** -3 * val, rel=1e-6)


@pytest.mark.parametrize("alpha", [0.75, 1.25, 1.5, 1.75])
def test_window_correction_1d_is_continued_zeta(alpha):
    # In grid units a = (A2 + A3) h^{d+alpha-2} equals, up to O(rho^-4), the
    # analytically continued lattice sum: zeta(alpha - 1) in 1D (it is the
    # regularised value of sum_{m>=1} m^{1-alpha}).
    h = 1.0
    a = cst.a2(1, alpha, h, 20 * h) + cst.a3(1, alpha, h, 20 * h)
    assert a == pytest.approx(special.zeta(alpha - 1), rel=1e-5)


@pytest.mark.parametrize("d,alpha", [(2, 0.5), (2, 1.5), (3, 1.0), (3, 1.9)])
def test_window_correction_is_negative_and_h_scaled(d, alpha):
    # A2 + A3 < 0 (Sec. 3.1) and A2 + A3 scales as h^{2-d-alpha} at fixed
    # rho = delta/h
    v1 = cst.a2(d, alpha, 1.0, 20.0) + cst.a3(d, alpha, 1.0, 20.0)
    h = 1.0 / 65
    v2 = cst.a2(d, alpha, h, 20 * h) + cst.a3(d, alpha, h, 20 * h)
    assert v1 < 0
    assert v2 == pytest.approx(v1 * h ** (2 - d - alpha), rel=1e-11)
    # and tends to Z_d(alpha - 2) / (2 d) (continued Epstein zeta)
    assert v1 == pytest.approx(cst.lattice_zeta(d, alpha - 2) / (2 * d), rel=1e-5)
