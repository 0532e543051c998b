"""Host logic of the GPU workloads (no GPU): the grid error estimate
(eq. rich) and the restriction of the finer grids to the coarse points."""

import numpy as np
import pytest

from paper_1802_03770_gb300 import inputs
from paper_1802_03770_gb300.workloads import _on_coarse, _rates


@pytest.mark.parametrize("d", [1, 2, 3])
def test_restriction_hits_the_coarse_points(d):
    nc = 7
    xc = inputs.grid_axes(nc, d)
    for k in (1, 2):
        n = 2 ** k * (nc + 1) - 1
        x = inputs.grid_axes(n, d)
        # the coordinate of every restricted point equals the coarse one
        grid = np.meshgrid(*x, indexing="ij")
        for ax in range(d):
            got = _on_coarse(grid[ax].ravel(), n, k, d)
            want = np.meshgrid(*xc, indexing="ij")[ax]
            assert np.array_equal(got, want)


@pytest.mark.parametrize("p", [0.5, 1.0, 2.0, 2.7])
def test_rates_of_an_exact_power_law(p):
    """Fields f_k = f* + h_k^p e (h halving) have R_2 = R_inf = p."""
    rng = np.random.default_rng(0)
    e = rng.standard_normal((5, 5))
    fstar = rng.standard_normal((5, 5))
    fields = [fstar + (0.1 / 2 ** k) ** p * e for k in range(3)]
    r = _rates(*fields)
    assert r["R2"] == pytest.approx(p, rel=1e-12)
    assert r["Rinf"] == pytest.approx(p, rel=1e-12)
