"""The learned preconditioner's alpha gate: band choice from validation
solves and the gate file (host logic, no GPU)."""

import math

from paper_1802_03770_gb300 import learned
from paper_1802_03770_gb300.api import read_gate


def _row(alpha, plain, learn):
    return {"alpha": alpha, "plain": {"iterations": plain}, "learned": {"iterations": learn}}


def test_band_enabled_only_where_learned_iterations_are_lower(tmp_path):
    # bands of width 0.5 on [0, 1.5): the network helps in the first band,
    # ties in the second (not enabled), hurts in the third
    rows = [_row(0.1, 50, 40), _row(0.3, 60, 44),
            _row(0.6, 30, 30), _row(0.9, 32, 32),
            _row(1.2, 20, 25)]
    flags, stats = learned.choose_gate(rows, 0.0, 1.5, 3)
    assert flags == [1, 0, 0]
    assert stats[0][2] == 2 and stats[0][3] == 55.0 and stats[0][4] == 42.0
    assert stats[2][2] == 1
    path = tmp_path / "gate.txt"
    learned.write_gate(str(path), flags, stats, "test", 0.0, 1.5)
    lo, hi, got = read_gate(str(path))
    assert (lo, hi, got) == (0.0, 1.5, [1, 0, 0])


def test_band_without_solves_stays_off():
    flags, stats = learned.choose_gate([_row(0.1, 10, 5)], 0.0, 1.0, 2)
    assert flags == [1, 0]
    assert stats[1][2] == 0 and math.isnan(stats[1][3])
