"""Selection oracle -- TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Pure-Python statements of the adaptive region's host logic, written from the
paper's description:

* variant ranges ``[BEGIN:END:STEP]`` (Section 3.1, "variants" clause) and
  the policy -> value mapping ``value = BEGIN + policy * STEP`` (Listings 4
  and 5, right-hand side);
* RoundRobin exploration and the "unique data point" count that triggers
  training (Section 2, the Apollo example: a point is unique when its
  features or its variant differ);
* label construction: for each feature vector, the fastest variant over the
  recorded executions (Section 2, "finds the fastest execution policies per
  feature values");
* the decision-tree classifier (Section 3.1, "model_type(dtree[, depth])",
  default depth 2) as exact greedy CART with Gini impurity;
* exhaustive argmin and the regret of a selection against it.

Readings where the paper is silent (tie-breaks, threshold placement, range
rounding) are stated on each function.
"""
from __future__ import annotations

import math
from fractions import Fraction

TIE_REL = 0.005  # means within 0.5 % of the best count as ties


# ------------------------------------------------------------ variant ranges
def expand_range(begin: float, end: float, step: float) -> list[float]:
    """Inclusive range [BEGIN:END:STEP] (Section 3.1): values BEGIN + i*STEP for
    i = 0 .. floor((END-BEGIN)/STEP + 1e-9).  Each value is computed from i,
    not by repeated addition, so float ranges like [0.0:1.0:0.1] keep END."""
    if not (step > 0) or end < begin:
        raise ValueError("range needs step > 0 and end >= begin")
    count = int(math.floor((end - begin) / step + 1e-9)) + 1
    return [begin + i * step for i in range(count)]


def policy_value(begin: float, step: float, policy: int) -> float:
    """Numeric variant value of a policy index (Listing 4: MIN + policy*STEP)."""
    return begin + policy * step


# ------------------------------------------------------------ exploration
def round_robin(call_index: int, num_variants: int) -> int:
    """Policy explored at the call_index-th query before training (Section 2:
    the runtime cycles through the policies)."""
    return call_index % num_variants


def unique_points(records) -> int:
    """Number of distinct (feature vector, variant) pairs among records given
    as (features tuple, variant, ms) (Section 2's uniqueness rule)."""
    return len({(tuple(f), int(v)) for f, v, _ in records})


# ------------------------------------------------------------ labels
def mean_table(records):
    """{features: {variant: mean ms}} over records (features, variant, ms)."""
    acc: dict = {}
    for f, v, ms in records:
        d = acc.setdefault(tuple(f), {})
        s = d.setdefault(int(v), [0.0, 0])
        s[0] += float(ms)
        s[1] += 1
    return {f: {v: s / n for v, (s, n) in d.items()} for f, d in acc.items()}


def best_variant(means: dict) -> int:
    """Fastest variant of a {variant: mean} table; means within 0.5 % of the
    minimum tie, and ties go to the lowest variant index."""
    m = min(means.values())
    return min(v for v, t in means.items() if t <= m * (1.0 + TIE_REL))


def labels(records):
    """Training set for the classifier: one (features, label) per distinct
    feature vector, label = fastest variant (Section 2), sorted by features."""
    tab = mean_table(records)
    return [(f, best_variant(tab[f])) for f in sorted(tab)]


def exhaustive_argmin(times) -> int:
    """Argmin of a per-variant mean-time list with the tie rule above."""
    return best_variant({v: t for v, t in enumerate(times)})


def regret(times, selected: int) -> float:
    """t(selected) / t(best) - 1 using the exhaustive table's mean times."""
    best = min(times)
    return times[selected] / best - 1.0


# ------------------------------------------------------------ CART
def _score(left_counts, nl, right_counts, nr) -> Fraction:
    """sum_c cL^2/nL + sum_c cR^2/nR; maximising it minimises the weighted
    Gini impurity nL*G(L) + nR*G(R).  Exact rational, so ties are exact."""
    return (Fraction(sum(c * c for c in left_counts.values()), nl)
            + Fraction(sum(c * c for c in right_counts.values()), nr))


def _majority(ys) -> int:
    cnt: dict = {}
    for y in ys:
        cnt[y] = cnt.get(y, 0) + 1
    top = max(cnt.values())
    return min(y for y, c in cnt.items() if c == top)


def cart_fit(X, y, max_depth: int = 2, samples=None, feature_draw=None):
    """Greedy CART classifier (Gini).

    Readings: candidate thresholds are midpoints (in float64) of consecutive
    distinct values of a feature; a sample goes left when x <= threshold; the
    split with the lowest weighted Gini wins, ties to the lowest feature index
    and then the lowest threshold; a node becomes a leaf at max_depth, when it
    is pure, or when no feature varies; a leaf predicts the majority label,
    ties to the lowest label.  Returns a list of nodes
    (feature, threshold, left, right, label); feature -1 marks a leaf.

    ``samples`` (default: every row once) is the multiset of row indices the
    tree is grown on; ``feature_draw()``, if given, is called once per split
    attempt and returns the candidate features for that node (random forest).
    """
    nodes = []

    def grow(idx, depth):
        me = len(nodes)
        nodes.append(None)
        ys = [y[i] for i in idx]
        if depth >= max_depth or len(set(ys)) <= 1 or len(idx) < 2:
            nodes[me] = (-1, 0.0, -1, -1, _majority(ys))
            return me
        best = None
        F = len(X[0])
        for f in (sorted(feature_draw()) if feature_draw else range(F)):
            vals = sorted({float(X[i][f]) for i in idx})
            for a in range(len(vals) - 1):
                thr = (vals[a] + vals[a + 1]) / 2.0
                lc, rc, nl, nr = {}, {}, 0, 0
                for i in idx:
                    if float(X[i][f]) <= thr:
                        lc[y[i]] = lc.get(y[i], 0) + 1
                        nl += 1
                    else:
                        rc[y[i]] = rc.get(y[i], 0) + 1
                        nr += 1
                s = _score(lc, nl, rc, nr)
                if best is None or s > best[0]:
                    best = (s, f, thr)
        if best is None:
            nodes[me] = (-1, 0.0, -1, -1, _majority(ys))
            return me
        _, f, thr = best
        li = [i for i in idx if float(X[i][f]) <= thr]
        ri = [i for i in idx if float(X[i][f]) > thr]
        left = grow(li, depth + 1)
        right = grow(ri, depth + 1)
        nodes[me] = (f, thr, left, right, _majority(ys))
        return me

    grow(list(range(len(y))) if samples is None else list(samples), 0)
    return nodes


# ------------------------------------------------------------ random forest
MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a 64-bit state advanced
    by the golden-ratio increment, output through two xor-shift-multiply
    rounds and a final xor-shift."""

    def __init__(self, seed: int):
        self.s = seed & MASK64

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & MASK64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def rfc_fit(X, y, ntrees: int, max_depth: int, seed: int):
    """Random forest (Section 3.1, model_type rfc with a tree count and a
    depth).  Reading: tree t is CART grown on a bootstrap sample (n indices
    next() mod n) and, at every split attempt in depth-first preorder, on
    mtry = max(1, floor(sqrt(F))) features drawn by a partial Fisher-Yates
    shuffle (position a swaps with a + next() mod (F - a)); one SplitMix64
    stream serves all trees in order."""
    rng = SplitMix64(seed)
    n, F = len(y), len(X[0])
    mtry = max(1, int(math.floor(math.sqrt(F))))

    def draw():
        feats = list(range(F))
        for a in range(mtry):
            b = a + rng.next() % (F - a)
            feats[a], feats[b] = feats[b], feats[a]
        return feats[:mtry]

    forest = []
    for _ in range(ntrees):
        samples = [rng.next() % n for _ in range(n)]
        forest.append(cart_fit(X, y, max_depth, samples=samples, feature_draw=draw))
    return forest


def rfc_predict(forest, x):
    """Majority vote of the trees, ties to the lowest label; returns (label,
    vote share)."""
    votes: dict = {}
    for t in forest:
        v = cart_predict(t, x)
        votes[v] = votes.get(v, 0) + 1
    top = max(votes.values())
    lab = min(v for v, c in votes.items() if c == top)
    return lab, top / len(forest)


def cart_predict(nodes, x) -> int:
    n = 0
    while nodes[n][0] >= 0:
        f, thr, left, right, _ = nodes[n]
        n = left if float(x[f]) <= thr else right
    return nodes[n][4]


def cart_depth(nodes) -> int:
    def d(n):
        f, _, left, right, _ = nodes[n]
        return 0 if f < 0 else 1 + max(d(left), d(right))

    return d(0)


def training_errors(predict, X, y) -> int:
    return sum(1 for xi, yi in zip(X, y) if predict(xi) != yi)
