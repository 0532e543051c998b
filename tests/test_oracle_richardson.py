"""The oracle against the paper's 2D grid error estimates (Table tab:2drich,
Sec. 4.2; eq. rich): rates of f = M g_1 (eq. test) and of the solution of
M u = 1 on the grids 255^2, 511^2, 1023^2, restricted to the common coarse
grid.

The u columns are reproduced to the printed two digits (checked here at
alpha = 1.5, the other two alphas on the GPU).  The f columns are not: the
oracle's rates are 2.77 / 2.51 / 2.25 against the printed 2.65 / 2.38 /
2.16, both above the second order of the consistency result (Theorem 1);
the window radius does not explain the gap (rho = 5 .. 40 gives 2.45 ..
2.6 at alpha = 1.5).  The f pin is therefore loose (0.2) and the u pin
tight (0.02)."""

import numpy as np
import pytest

from oracle import solvers
from oracle.operator import Plan
from paper_1802_03770_gb300 import inputs

GRIDS = (255, 511, 1023)


def rates(c, m, f):
    out = []
    for p in (2, np.inf):
        a = np.linalg.norm((f - m).ravel(), p)
        b = np.linalg.norm((m - c).ravel(), p)
        out.append((np.log(a) - np.log(b)) / np.log(0.5))
    return out


def coarse(v, k):
    s = 2 ** k
    return v[s - 1::s, s - 1::s]


def paper(golden, field, alpha):
    for t, d, fld, a, r2, rinf in golden("table_richardson.txt"):
        if t == 1 and fld == field and abs(a - alpha) < 1e-9:
            return r2, rinf
    raise KeyError(alpha)


@pytest.mark.parametrize("alpha", [1.25, 1.5, 1.75])
def test_apply_rates_table_2drich(golden, alpha):
    fs = []
    for k, n in enumerate(GRIDS):
        p = Plan(2, n, 1.0 / (n + 1), alpha)
        fs.append(coarse(p.apply(inputs.cosine_product(n, 2, (1, 1))), k))
    r2, rinf = rates(*fs)
    p2, pinf = paper(golden, 1, alpha)
    assert r2 > 2.0 and rinf > 2.0
    assert abs(r2 - p2) <= 0.2 and abs(rinf - pinf) <= 0.2


@pytest.mark.slow
def test_solution_rates_table_2drich_alpha_1_5(golden):
    us = []
    for k, n in enumerate(GRIDS):
        p = Plan(2, n, 1.0 / (n + 1), 1.5)
        u, _, ok, _ = solvers.solve_elliptic(p, np.ones(p.n), tol=1e-11, maxit=2000)
        assert ok
        us.append(coarse(u, k))
    r2, rinf = rates(*us)
    p2, pinf = paper(golden, 0, 1.5)
    assert abs(r2 - p2) <= 0.02 and abs(rinf - pinf) <= 0.02
