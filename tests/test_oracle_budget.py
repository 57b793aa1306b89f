"""Pins of the entry-budget threshold of the oracle (paper, Methods, "Other
algorithmic improvements": fitting the posterior matrices into a given amount
of memory by keeping fewer entries).

The oracle returns the smallest threshold, in the precision the entries are
compared in, whose kept entries fit the budget.  It is checked against an
exhaustive search over every threshold at which the kept count can change
(the values themselves, one unit above each, and theta), on small inputs with
many ties, and against hand-worked cases."""
import numpy as np
import pytest

import oracle


def _brute(values, theta, n_keep, dtype):
    v = np.asarray(values, dtype=dtype)
    cands = {dtype(theta)}
    for x in v:
        cands.add(dtype(x))
        cands.add(np.nextafter(dtype(x), dtype(np.inf)))
    ok = [c for c in cands if c >= dtype(theta) and np.count_nonzero(v >= c) <= n_keep]
    return min(ok)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_matches_exhaustive_search(dtype):
    rng = np.random.default_rng(11)
    theta = 0.01
    for trial in range(300):
        n = int(rng.integers(0, 12))
        levels = [None, 2, 3, 5][trial % 4]
        if levels is None:
            v = theta + (1 - theta) * rng.random(n)
        else:
            v = theta + (1 - theta) * rng.integers(0, levels, n) / levels
        v = v.astype(dtype)
        for n_keep in range(0, n + 2):
            t = oracle.budget_threshold(v, theta, n_keep, dtype)
            assert t == _brute(v, theta, n_keep, dtype), (trial, n_keep)
            assert np.count_nonzero(v >= t) <= n_keep
            assert t >= dtype(theta)


def test_hand_cases():
    v = np.array([0.5, 0.4, 0.4, 0.3], dtype=np.float32)
    f = np.float32
    # room for 2: the third largest (0.4) and its tie go; only 0.5 stays
    t = oracle.budget_threshold(v, 0.1, 2, f)
    assert t == np.nextafter(f(0.4), f(1)) and np.count_nonzero(v >= t) == 1
    # room for 3: 0.3 goes
    t = oracle.budget_threshold(v, 0.1, 3, f)
    assert t == np.nextafter(f(0.3), f(1)) and np.count_nonzero(v >= t) == 3
    # room for all: the threshold stays
    assert oracle.budget_threshold(v, 0.1, 4, f) == f(0.1)
    assert oracle.budget_threshold(v, 0.1, 100, f) == f(0.1)
    # room for none: everything goes
    t = oracle.budget_threshold(v, 0.1, 0, f)
    assert t == np.nextafter(f(0.5), f(1)) and np.count_nonzero(v >= t) == 0
    # no entries at all
    assert oracle.budget_threshold(np.zeros(0, dtype=f), 0.25, 0, f) == f(0.25)


def test_precision_of_the_comparison():
    """The threshold is the float (or double) one unit above the cut value,
    not a rounded decimal."""
    x = 0.1234567
    t32 = oracle.budget_threshold(np.array([x, x / 2], np.float32), 0.01, 1, np.float32)
    t64 = oracle.budget_threshold(np.array([x, x / 2], np.float64), 0.01, 1, np.float64)
    assert t32 == np.nextafter(np.float32(x / 2), np.float32(1))
    assert t64 == np.nextafter(x / 2, 1.0)
    assert t32 != t64
