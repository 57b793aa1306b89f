"""Pins of the guide-tree oracle (weighted UPGMA, paper Methods stage II).

The oracle is checked against facts fixed by the method itself, not by
re-typing it: an ultrametric distance matrix is reproduced exactly (every
join at its lowest common ancestor, at that ancestor's height), a
hand-computed four-leaf case separates weighted from unweighted averaging,
and equal distances follow the stated tie rule."""
import numpy as np
import pytest

import oracle


def _random_ultrametric(rng, k):
    """A random rooted binary tree over k leaves with distinct internal
    heights; d(a, b) = 2 * height(lowest common ancestor).  Returns the
    matrix and the set of (frozenset of leaves, height) of internal nodes."""
    clusters = [frozenset([i]) for i in range(k)]
    heights = np.sort(rng.uniform(0.1, 10.0, size=k - 1))
    nodes = []
    D = np.zeros((k, k))
    for h in heights:
        a, b = rng.choice(len(clusters), size=2, replace=False)
        A, B = clusters[a], clusters[b]
        for x in A:
            for y in B:
                D[x, y] = D[y, x] = 2.0 * h
        merged = A | B
        nodes.append((merged, h))
        clusters = [c for i, c in enumerate(clusters) if i not in (a, b)] + [merged]
    return D, set(nodes)


def _leaf_sets(merges, k):
    members = {i: frozenset([i]) for i in range(k)}
    out = []
    for s, (a, b) in enumerate(merges):
        members[k + s] = members[int(a)] | members[int(b)]
        out.append(members[k + s])
    return out


@pytest.mark.parametrize("k", [2, 3, 7, 40])
def test_ultrametric_tree_is_recovered(k):
    rng = np.random.default_rng(k)
    D, nodes = _random_ultrametric(rng, k)
    r = oracle.guide_tree(D)
    got = set(zip(_leaf_sets(r["merges"], k), r["heights"].tolist()))
    assert got == {(c, h) for c, h in nodes}


def test_weighted_average_hand_example():
    """A, B, C, D = slots 0..3.  Join A, B at 2 (height 1): d(AB, C) =
    (4 + 6) / 2 = 5, d(AB, D) = (10 + 10) / 2 = 10.  Join AB, C at 5 (height
    2.5): d(ABC, D) = (10 + 8) / 2 = 9 (height 4.5).  Unweighted UPGMA would
    give (2 * 10 + 8) / 3 = 9.33 here."""
    D = np.array([[0, 2, 4, 10],
                  [2, 0, 6, 10],
                  [4, 6, 0, 8],
                  [10, 10, 8, 0]], dtype=float)
    r = oracle.guide_tree(D)
    assert r["merges"].tolist() == [[0, 1], [4, 2], [5, 3]]
    assert r["heights"].tolist() == [1.0, 2.5, 4.5]


def test_tie_rule():
    """Equal distances: the smallest slot i, then the smallest j; the joined
    cluster takes slot i."""
    D = np.ones((4, 4)) - np.eye(4)
    r = oracle.guide_tree(D)
    assert r["merges"].tolist() == [[0, 1], [4, 2], [5, 3]]
    assert r["heights"].tolist() == [0.5, 0.5, 0.5]


def test_merges_form_a_binary_tree():
    rng = np.random.default_rng(3)
    k = 25
    A = rng.random((k, k))
    D = (A + A.T) / 2
    np.fill_diagonal(D, 0)
    r = oracle.guide_tree(D)
    ids = r["merges"].ravel().tolist()
    assert sorted(ids) == list(range(2 * k - 2)), "every node but the root is joined exactly once"
    for s, (a, b) in enumerate(r["merges"]):
        assert a < k + s and b < k + s, "a cluster is joined after it is formed"


def test_rejects_bad_shapes():
    with pytest.raises(ValueError):
        oracle.guide_tree(np.zeros((1, 1)))
    with pytest.raises(ValueError):
        oracle.guide_tree(np.zeros((3, 4)))
