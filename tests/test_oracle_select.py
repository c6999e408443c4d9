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


# ------------------------------------------------------------ forest worked example
# A 2-tree, depth-2 forest on 6 rows and 4 features (mtry = floor(sqrt 4) = 2),
# seed 0, worked out by hand from the SplitMix64 stream.  Every draw below is
# a literal derived from the stream, and every split from exact Gini scores
# (score = sum_c cL^2/nL + sum_c cR^2/nR, higher is better).
RFC_X = [[1.0, 2.0, 3.0, 3.0], [0.0, 0.0, 3.0, 3.0], [0.0, 1.0, 3.0, 1.0],
         [1.0, 3.0, 1.0, 1.0], [2.0, 2.0, 0.0, 0.0], [3.0, 3.0, 3.0, 2.0]]
RFC_Y = [2, 0, 1, 2, 0, 0]
# the first 20 outputs of SplitMix64 from state 0 (0..7 also in the golden file)
RFC_STREAM = [
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f, 0xf88bb8a8724c81ec,
    0x1b39896a51a8749b, 0x53cb9f0c747ea2ea, 0x2c829abe1f4532e1, 0xc584133ac916ab3c,
    0x3ee5789041c98ac3, 0xf3b8488c368cb0a6, 0x657eecdd3cb13d09, 0xc2d326e0055bdef6,
    0x8621a03fe0bbdb7b, 0x8e1f7555983aa92f, 0xb54e0f1600cc4d19, 0x84bb3f97971d80ab,
    0x7d29825c75521255, 0xc3cf17102b7f7f86, 0x3466e9a083914f64, 0xd81a8d2b5a4485ac,
]
# Tree 1 consumes outputs 0..9:
#   bootstrap = outputs 0..5 mod 6 = [1, 0, 1, 4, 1, 0] (row 1 x3, row 0 x2, row 4)
#   root draw: output 6 mod 4 = 1 swaps slots 0,1 -> [1,0,2,3]; 1 + output 7 mod 3
#     = 3 swaps slots 1,3 -> [1,3,2,0]: features {1, 3}.  Feature 1 at 1.0 scores
#     9/3 + 5/3 = 14/3, feature 3 at 1.5 scores 1 + 13/5 = 18/5: split (1, 1.0).
#   left child = row 1 x3, pure: a leaf, no draw.
#   right child = row 0 x2 (label 2), row 4 (label 0): draw outputs 8, 9 ->
#     [3,1,2,0] -> [3,0,2,1]: features {0, 3}; both score 4/2 + 1 = 3, the tie
#     goes to feature 0: split (0, 1.5).  (A draw made once per tree would offer
#     {1, 3} here, where feature 1 does not vary: split (3, 1.5) instead.)
# Tree 2 consumes outputs 10..19:
#   bootstrap = outputs 10..15 mod 6 = [1, 4, 3, 3, 5, 1]
#   root draw: outputs 16, 17 -> [1,0,2,3] -> [1,3,2,0]: features {1, 3}.
#     Feature 1 at 2.5 and feature 3 at 1.5 both score 3 + 5/3 = 14/3 (best);
#     the tie goes to feature 1: split (1, 2.5).
#   left child = row 1 x2, row 4: all label 0, a leaf.
#   right child = row 3 x2 (label 2), row 5 (label 0): outputs 18, 19 ->
#     [0,1,2,3] -> [0,2,1,3]: features {0, 2}, both score 3: split (0, 2.0).
RFC_BOOT = [[1, 0, 1, 4, 1, 0], [1, 4, 3, 3, 5, 1]]
RFC_DRAWS = [[[1, 3], [0, 3]], [[1, 3], [0, 2]]]
RFC_FOREST = [
    [(1, 1.0, 1, 2, 0), (-1, 0.0, -1, -1, 0), (0, 1.5, 3, 4, 2), (-1, 0.0, -1, -1, 2),
     (-1, 0.0, -1, -1, 0)],
    [(1, 2.5, 1, 2, 0), (-1, 0.0, -1, -1, 0), (0, 2.0, 3, 4, 2), (-1, 0.0, -1, -1, 2),
     (-1, 0.0, -1, -1, 0)],
]


def test_rfc_stream_and_derived_draws():
    r = select.SplitMix64(0)
    assert [r.next() for _ in RFC_STREAM] == RFC_STREAM
    # the literal bootstrap indices and subsets restate the stream arithmetic
    assert [o % 6 for o in RFC_STREAM[0:6]] == RFC_BOOT[0]
    assert [o % 6 for o in RFC_STREAM[10:16]] == RFC_BOOT[1]


def test_rfc_worked_example_forest():
    forest = select.rfc_fit(RFC_X, RFC_Y, ntrees=2, max_depth=2, seed=0)
    assert forest == RFC_FOREST
    # the same trees from the (separately pinned) CART with the hand-derived
    # bootstrap samples and per-split feature subsets
    for t in range(2):
        draws = iter(RFC_DRAWS[t])
        tree = select.cart_fit(RFC_X, RFC_Y, 2, samples=RFC_BOOT[t], feature_draw=lambda: next(draws))
        assert tree == RFC_FOREST[t]
        assert next(draws, None) is None  # exactly one draw per split attempt


def _mutated_rfc(old: str, new: str):
    """rfc_fit with one planted mistake (a textual edit of its source)."""
    import inspect
    import textwrap

    src = textwrap.dedent(inspect.getsource(select.rfc_fit))
    assert old in src, old
    ns = dict(vars(select))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["rfc_fit"]


@pytest.mark.parametrize("old,new", [
    ("for _ in range(n)]", "for _ in range(n - 1)]"),                 # bootstrap of n-1
    ("rng.next() % n ", "rng.next() % (n - 1) "),                     # indices mod n-1
    ("feature_draw=draw", "feature_draw=(lambda s=draw(): (lambda: s))()"),  # one draw per tree
    ("for a in range(mtry):", "for a in range(F - 1):"),              # full shuffle
    ("int(math.floor(math.sqrt(F)))", "F"),                           # every feature
])
def test_rfc_worked_example_rejects_planted_mistakes(old, new):
    forest = _mutated_rfc(old, new)(RFC_X, RFC_Y, ntrees=2, max_depth=2, seed=0)
    assert forest != RFC_FOREST
