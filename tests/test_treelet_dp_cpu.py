"""The treelet restructuring's optimisation step, restated on the CPU (no
GPU): for a treelet of k leaf boxes (the kernel's treelets have at most 7;
up to 8 here), the dynamic programme over leaf
subsets -- each subset's best split into the part holding its lowest leaf
and the rest, smallest subsets first -- finds the binary tree with the
smallest summed surface area of its internal nodes.  Checked against brute
force over every binary tree on the same leaves (135,135 trees for k = 8)."""
import itertools

import numpy as np
import pytest


def _area(lo, hi):
    e = np.maximum(hi - lo, 0.0)
    return e[0] * e[1] + e[1] * e[2] + e[2] * e[0]


def _subset_area(boxes, S):
    idx = [i for i in range(len(boxes)) if (S >> i) & 1]
    lo = np.min([boxes[i][0] for i in idx], 0)
    hi = np.max([boxes[i][1] for i in idx], 0)
    return _area(lo, hi)


def dp_cost(boxes):
    """The kernel's programme: cost[S] = area(S) + min over splits (Q, S ^ Q),
    Q holding the lowest leaf of S and Q != S; single leaves cost 0."""
    k = len(boxes)
    full = (1 << k) - 1
    cost = np.zeros(full + 1)
    for S in sorted(range(1, full + 1), key=lambda s: bin(s).count("1")):
        if S & (S - 1) == 0:
            continue
        low = S & -S
        rest = S ^ low
        best = np.inf
        sub = (rest - 1) & rest
        while True:
            Q = low | sub
            best = min(best, cost[Q] + cost[S ^ Q])
            if sub == 0:
                break
            sub = (sub - 1) & rest
        cost[S] = _subset_area(boxes, S) + best
    return cost[full]


def _trees(items):
    """Every binary tree (nested pairs) over the tuple of leaf indices."""
    if len(items) == 1:
        yield items[0]
        return
    first, rest = items[0], items[1:]
    # split into the part with the first leaf and a non-empty rest
    for r in range(0, len(rest)):
        for comb in itertools.combinations(rest, r):
            left = (first,) + comb
            right = tuple(x for x in rest if x not in comb)
            for a in _trees(left):
                for b in _trees(right):
                    yield (a, b)


def _tree_cost(t, boxes):
    if isinstance(t, int):
        return 0.0, boxes[t][0], boxes[t][1]
    ca, la, ha = _tree_cost(t[0], boxes)
    cb, lb, hb = _tree_cost(t[1], boxes)
    lo, hi = np.minimum(la, lb), np.maximum(ha, hb)
    return ca + cb + _area(lo, hi), lo, hi


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7, 8])
def test_programme_finds_the_best_tree(k):
    rng = np.random.default_rng(k)
    for _ in range({7: 4, 8: 1}.get(k, 20)):
        c = rng.uniform(-1, 1, (k, 3))
        e = rng.uniform(0.0, 0.5, (k, 3)) * rng.choice([0.0, 1.0], (k, 3), p=[0.1, 0.9])   # some flat boxes
        boxes = [(c[i] - e[i], c[i] + e[i]) for i in range(k)]
        brute = min(_tree_cost(t, boxes)[0] for t in _trees(tuple(range(k))))
        assert dp_cost(boxes) == pytest.approx(brute, rel=1e-12)


def test_tree_count_is_the_double_factorial():
    """The brute force enumerates each binary tree once: (2k - 3)!! trees."""
    for k, count in ((3, 3), (4, 15), (5, 105), (6, 945), (7, 10395)):
        assert sum(1 for _ in _trees(tuple(range(k)))) == count
