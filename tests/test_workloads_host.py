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


class _FakePlan:
    """Stands in for api.Plan in the batch tuner: records the launch shapes
    the tuner sets; its autotune() returns a fixed per-plan choice."""

    def __init__(self, tuned, shape, row_len):
        self.tuned, self.tuned_shape, self.row_len = tuned, shape, row_len
        self.tiles, self.shape = [0] * 6, 0

    def autotune(self):
        self.tiles, self.shape = list(self.tuned), self.tuned_shape
        return list(self.tuned)

    def row_shape(self):
        return self.shape

    def set_tiles(self, tx):
        self.tiles = list(tx)

    def set_row_shape(self, s):
        self.shape = s

    def describe(self):
        return {"fft_len": (self.row_len, self.row_len)}


@pytest.mark.parametrize("fastest", ["per_plan", "widest", "widest_rows256x8"])
def test_tune_batch_keeps_the_fastest_configuration(monkeypatch, fastest):
    """tune_batch times every candidate on the batched solve and leaves the
    plans in the fastest one (per-plan tiles and shapes restored, or the
    widest tiles with one row shape on every plan)."""
    import sys
    import types
    from paper_1802_03770_gb300 import workloads

    plans = [_FakePlan([2, 0, 0, 1, 0, 0], 1, 512), _FakePlan([4, 0, 0, 2, 0, 0], 0, 1024)]
    cost = {"per_plan": 3.0, "widest": 2.0, "widest_rows256x8": 2.5}
    cost[fastest] = 1.0
    clock = {"t": 0.0}

    def config():
        if any(p.tiles != [0] * 6 for p in plans):
            return "per_plan"
        return "widest_rows256x8" if all(p.shape == 1 for p in plans) else "widest"

    def fake_solve(ps, fs, tol, mode):
        clock["t"] += cost[config()]

    monkeypatch.setattr(workloads, "solve_batched", fake_solve)
    monkeypatch.setattr(workloads.time, "perf_counter", lambda: clock["t"])
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    choice, times = workloads.tune_batch(plans, [None, None], mode=0, reps=2)
    assert choice == fastest
    assert set(times) == {"per_plan", "widest", "widest_rows256x8"}
    assert config() == fastest
    if fastest == "per_plan":
        assert [p.tiles for p in plans] == [[2, 0, 0, 1, 0, 0], [4, 0, 0, 2, 0, 0]]
        assert [p.shape for p in plans] == [1, 0]


def test_tune_batch_skips_the_256x8_rows_for_short_rows(monkeypatch):
    import sys
    import types
    from paper_1802_03770_gb300 import workloads
    plans = [_FakePlan([2, 0, 0, 1, 0, 0], 0, 128), _FakePlan([4, 0, 0, 1, 0, 0], 0, 512)]
    monkeypatch.setattr(workloads, "solve_batched", lambda ps, fs, tol, mode: None)
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    _, times = workloads.tune_batch(plans, [None, None], mode=0, reps=1)
    assert set(times) == {"per_plan", "widest"}
