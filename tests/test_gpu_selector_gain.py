"""What the learned selector gains (GPU): on held-out SpMV matrices the
device-trained MLP picks variants whose regret against exhaustive profiling
is well below that of the paper's depth-2 decision tree and of the fixed
default variant, both trained or fixed on the same profiling records."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu


def test_mlp_beats_tree_and_default_on_held_out_matrices():
    # 400 training matrices: with 160 the two selectors' regrets overlapped
    # from run to run (3.3-4.2 % against 3.4 %); with 400 the MLP's is about
    # half the tree's (1.5 % against 2.7 %)
    r = bench.spmv_study(n_train=400, n_test=80, rows_max=1e6, epochs=300)["selection"]
    assert r["mlp_mean_regret_pct"] <= 8.0
    assert r["mlp_mean_regret_pct"] < r["dtree_mean_regret_pct"]
    assert r["mlp_mean_regret_pct"] < r["default_mean_regret_pct"] / 10
    # the aggregate rate is dominated by the largest matrices, where both
    # selectors mostly pick the same variant or two within a few percent of
    # each other (merge path, binned, vector-8): the MLP within 2 % or better
    assert r["mlp_gbs"] >= 0.98 * r["dtree_gbs"] and r["mlp_gbs"] > 2 * r["default_gbs"]
