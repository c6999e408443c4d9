"""bench.py's implementation of the paper's evaluation protocol (Section 4.1)
on CPU: K-fold Adaptive-25/50/75, Adaptive-100 and Static,Best on synthetic
profile tables whose answers are known (host models only: the depth-2 tree
and the single best variant)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _table(n=40, V=3):
    """Feature x in 1..n; variant 0 is fastest for x <= 20 (1 ms against
    2 ms), variant 2 for x > 20; variant 1 is always 1.5 ms."""
    table = []
    for x in range(1, n + 1):
        ms = [1.0, 1.5, 2.0] if x <= 20 else [2.0, 1.5, 1.0]
        table.append(([float(x)], ms[:V]))
    return table


def test_tree_learns_a_threshold_and_static_best_pays_for_one_variant():
    table = _table()
    res = bench.kfold_protocol(table, 3, 1, epochs=1, shuffles=3, models=("dtree", "static_best"))
    # one threshold separates the two regimes: no regret once trained on all points
    assert res["dtree"]["adaptive_100"] == pytest.approx(0.0)
    # a single variant is twice as slow on half the points or 1.5x on all:
    # variant 1 (50 %) is the best single choice in total; regret 50 %
    assert res["static_best"]["adaptive_100"] == pytest.approx(50.0)
    for f in (25, 50, 75):
        assert 0.0 <= res["dtree"][f"adaptive_{f}"] <= res["static_best"][f"adaptive_{f}"] + 1e-9
        # Static,Best on any training subset picks variant 1 whenever both regimes are present
        assert res["static_best"][f"adaptive_{f}"] >= 50.0 - 1e-9


def test_single_regime_has_no_regret_for_either_model():
    table = [([float(x)], [1.0, 3.0]) for x in range(1, 17)]
    res = bench.kfold_protocol(table, 2, 1, epochs=1, shuffles=2, models=("dtree", "static_best"))
    for kind in ("dtree", "static_best"):
        for key, v in res[kind].items():
            assert v == pytest.approx(0.0), (kind, key)
