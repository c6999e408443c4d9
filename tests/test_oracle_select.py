"""Pins of the selection oracle: paper-printed ranges and defaults, brute
force over small decision trees, and closed-form label cases (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle import select

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "variant_ranges.json")))


@pytest.mark.parametrize("case", GOLD["ranges"])
def test_paper_ranges(case):
    vals = select.expand_range(case["begin"], case["end"], case["step"])
    if "values" in case:
        assert vals == case["values"]
    else:
        assert len(vals) == case["count"]
        assert vals[0] == case["first"]
        assert vals[-1] == pytest.approx(case["last"], abs=1e-12)


def test_policy_value_listing4():
    vals = select.expand_range(64, 1024, 64)
    assert [select.policy_value(64, 64, p) for p in range(16)] == vals


def test_range_rejects_bad_step():
    with pytest.raises(ValueError):
        select.expand_range(1, 0, 1)
    with pytest.raises(ValueError):
        select.expand_range(0, 1, 0)


def test_round_robin_cycles_all_policies():
    V = GOLD["apollo_example"]["num_policies"]
    seq = [select.round_robin(k, V) for k in range(6)]
    assert seq == [0, 1, 0, 1, 0, 1]


def test_unique_points_counts_feature_variant_pairs():
    recs = [((1.0,), 0, 2.0), ((1.0,), 0, 3.0), ((1.0,), 1, 1.0), ((2.0,), 0, 1.0)]
    assert select.unique_points(recs) == 3


def test_labels_pick_fastest_mean_with_ties_to_lowest():
    recs = [((8.0,), 0, 1.0), ((8.0,), 0, 3.0), ((8.0,), 1, 1.5), ((8.0,), 2, 2.2),
            ((9.0,), 0, 1.003), ((9.0,), 1, 1.0), ((9.0,), 2, 0.999)]
    lab = dict(select.labels(recs))
    assert lab[(8.0,)] == 1          # means 2.0, 1.5, 2.2
    assert lab[(9.0,)] == 0          # all within 0.5 % of 0.999: lowest index


def test_exhaustive_argmin_and_regret():
    t = [3.0, 1.0, 2.0]
    assert select.exhaustive_argmin(t) == 1
    assert select.regret(t, 1) == 0.0
    assert select.regret(t, 2) == pytest.approx(1.0)


# ------------------------------------------------------------- CART
def _gini_cost(groups):
    """sum over groups of n * Gini(group), as a float."""
    tot = 0.0
    for ys in groups:
        n = len(ys)
        if n == 0:
            continue
        cnt = np.bincount(ys)
        tot += n * (1.0 - np.sum((cnt / n) ** 2))
    return tot


def _all_splits(X, idx):
    F = X.shape[1]
    for f in range(F):
        vals = sorted(set(X[idx, f].tolist()))
        for a in range(len(vals) - 1):
            yield f, (vals[a] + vals[a + 1]) / 2.0


def _best_tree_errors(X, y, depth):
    """Fewest training errors over every tree of the given depth whose
    thresholds are midpoints (exhaustive enumeration)."""
    def best(idx, d):
        ys = y[idx]
        maj = np.bincount(ys).max() if len(ys) else 0
        e = len(ys) - maj
        if d == 0 or e == 0:
            return e
        for f, t in _all_splits(X, idx):
            li = idx[X[idx, f] <= t]
            ri = idx[X[idx, f] > t]
            e = min(e, best(li, d - 1) + best(ri, d - 1))
        return e
    return best(np.arange(len(y)), depth)


@pytest.mark.parametrize("seed", range(12))
def test_cart_root_is_the_best_gini_split_and_errors_bounded(seed):
    r = np.random.Generator(np.random.PCG64(100 + seed))
    n = int(r.integers(4, 13))
    X = r.integers(0, 5, (n, 2)).astype(np.float32)
    y = r.integers(0, 3, n)
    tree = select.cart_fit(X.tolist(), y.tolist(), max_depth=2)
    f, thr, _, _, _ = tree[0]
    if len(set(y.tolist())) > 1 and f >= 0:
        costs = []
        for ff, t in _all_splits(X, np.arange(n)):
            costs.append((_gini_cost([y[X[:, ff] <= t], y[X[:, ff] > t]]), ff, t))
        best_cost = min(c for c, _, _ in costs)
        mine = _gini_cost([y[X[:, f] <= thr], y[X[:, f] > thr]])
        assert mine == pytest.approx(best_cost, abs=1e-12)
        # first in (feature, threshold) order among the optimal ones
        first = min((ff, t) for c, ff, t in costs if abs(c - best_cost) <= 1e-12)
        assert (f, thr) == first
    errs = select.training_errors(lambda x: select.cart_predict(tree, x), X.tolist(), y.tolist())
    assert errs >= _best_tree_errors(X, y, 2)
    assert select.cart_depth(tree) <= 2


def test_cart_separable_single_threshold():
    X = [[float(v)] for v in (32, 64, 128, 256, 384, 512)]
    y = [0, 0, 0, 1, 1, 1]
    tree = select.cart_fit(X, y, max_depth=2)
    assert tree[0][:2] == (0, 192.0)
    assert [select.cart_predict(tree, x) for x in X] == y
    assert select.cart_depth(tree) == 1


def test_cart_depth_two_solves_two_thresholds():
    # three classes on one feature need two levels
    X = [[float(v)] for v in range(9)]
    y = [0, 0, 0, 1, 1, 1, 2, 2, 2]
    tree = select.cart_fit(X, y, max_depth=2)
    assert select.training_errors(lambda x: select.cart_predict(tree, x), X, y) == 0
    stump = select.cart_fit(X, y, max_depth=1)
    assert select.training_errors(lambda x: select.cart_predict(stump, x), X, y) == 3


def test_cart_constant_features_give_majority_leaf():
    tree = select.cart_fit([[1.0, 2.0]] * 5, [2, 1, 1, 2, 0], max_depth=2)
    assert tree == [(-1, 0.0, -1, -1, 1)]


# ------------------------------------------------------------- random forest
def test_splitmix64_known_outputs():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")))
    r = select.SplitMix64(g["seed"])
    assert [r.next() for _ in g["outputs"]] == [int(h, 16) for h in g["outputs"]]


def test_rfc_trees_respect_depth_and_vote():
    rng = np.random.Generator(np.random.PCG64(7))
    X = rng.integers(0, 6, (30, 3)).astype(np.float32).tolist()
    y = [int(a > 2) + 2 * int(b > 3) for a, b, _ in X]
    forest = select.rfc_fit(X, y, ntrees=25, max_depth=3, seed=11)
    assert len(forest) == 25 and all(select.cart_depth(t) <= 3 for t in forest)
    labs = set(y)
    for x in X:
        lab, share = select.rfc_predict(forest, x)
        assert lab in labs and 0 < share <= 1
    acc = np.mean([select.rfc_predict(forest, x)[0] == t for x, t in zip(X, y)])
    assert acc >= 0.8


def test_rfc_single_feature_bootstrap_of_all_identical_rows():
    # one distinct row: every bootstrap sample is that row, every tree a leaf
    forest = select.rfc_fit([[2.0, 5.0]] * 4, [3, 3, 3, 3], ntrees=3, max_depth=2, seed=1)
    assert forest == [[(-1, 0.0, -1, -1, 3)]] * 3
    assert select.rfc_predict(forest, [0.0, 0.0]) == (3, 1.0)


def test_rfc_vote_ties_go_to_lowest_label():
    forest = [[(-1, 0.0, -1, -1, 4)], [(-1, 0.0, -1, -1, 1)]]
    assert select.rfc_predict(forest, [0.0]) == (1, 0.5)
