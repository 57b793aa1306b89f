"""Pins of the selective-consistency oracle (paper, Methods, stage III and
"Selective consistency").

  * tree distances against a brute force over leaf sets and against the
    closed form of a caterpillar tree;
  * the relaxation against an element-wise quadruple loop (an independent
    writing of the same sum) on tiny random inputs, with and without
    selectivity and amplification;
  * invariants: a pair with no selected third sequence keeps its matrix; with
    identity matrices everything stays the identity; swapping the roles of x
    and y transposes the result; T = k admits every third sequence and h = 1
    gives the plain (ProbCons) average."""
import itertools

import numpy as np
import pytest

import oracle


def _random_merges(rng, k):
    slots = list(range(k))
    merges = []
    nxt = k
    while len(slots) > 1:
        i, j = sorted(rng.choice(len(slots), 2, replace=False).tolist())
        a, b = slots[i], slots[j]
        merges.append((a, b))
        slots.pop(j)
        slots[i] = nxt
        nxt += 1
    return np.array(merges)


def _leaves(merges, k, node):
    if node < k:
        return {node}
    a, b = merges[node - k]
    return _leaves(merges, k, int(a)) | _leaves(merges, k, int(b))


def test_tree_distance_brute_force():
    rng = np.random.default_rng(3)
    for k in (2, 3, 5, 9, 17):
        merges = _random_merges(rng, k)
        d = oracle.tree_distances(merges, k)
        nodes = [_leaves(merges, k, n) for n in range(2 * k - 1)]
        for x in range(k):
            for y in range(k):
                if x == y:
                    assert d[x, y] == 1
                    continue
                best = min(len(L) for L in nodes if x in L and y in L)
                assert d[x, y] == best


def test_tree_distance_caterpillar():
    """((((0,1),2),3),...): d(x, y) = max(x, y) + 1 for x != y, min >= 1."""
    k = 8
    merges = [(0, 1)] + [(k + s, s + 2) for s in range(k - 2)]
    d = oracle.tree_distances(merges, k)
    for x in range(k):
        for y in range(k):
            if x != y:
                assert d[x, y] == max(x, y, 1) + 1


def _random_S(rng, lens, density=0.5):
    k = len(lens)
    S = {}
    for a in range(k):
        for b in range(a + 1, k):
            M = rng.random((lens[a], lens[b])) * (rng.random((lens[a], lens[b])) < density)
            S[(a, b)] = M
    return S


def _brute(S, lens, merges, T, h, n_max, theta):
    """The same definition written element by element."""
    k = len(lens)
    d = oracle.tree_distances(merges, k)

    def el(a, b, i, j):
        return S[(a, b)][i, j] if a < b else S[(b, a)][j, i]

    out = {}
    for x, y in itertools.combinations(range(k), 2):
        Z = [z for z in range(k) if z not in (x, y) and d[x, z] <= T and d[z, y] <= T]
        hxy = 1.0 + (h - 1.0) * min(len(Z), n_max) / n_max
        R = np.zeros((lens[x], lens[y]))
        for i in range(lens[x]):
            for j in range(lens[y]):
                v = 2.0 * hxy * el(x, y, i, j)
                for z in Z:
                    for t in range(lens[z]):
                        v += el(x, z, i, t) * el(z, y, t, j)
                v /= 2.0 + len(Z)
                R[i, j] = v if v >= theta else 0.0
        out[(x, y)] = R
    return out


@pytest.mark.parametrize("T,h,n_max", [(100, 1.0, 200), (3, 3.0, 200), (4, 3.0, 2), (2, 2.0, 1)])
def test_relaxation_matches_elementwise_sum(T, h, n_max):
    rng = np.random.default_rng(T * 7 + n_max)
    k = 6
    lens = [int(v) for v in rng.integers(1, 5, k)]
    merges = _random_merges(rng, k)
    S = _random_S(rng, lens)
    got, nz = oracle.consistency(S, lens, merges, T=T, h=h, n_max=n_max, theta=0.05)
    exp = _brute(S, lens, merges, T, h, n_max, 0.05)
    for key in exp:
        np.testing.assert_allclose(got[key], exp[key], rtol=1e-13, atol=1e-15)


def test_no_selected_sequence_keeps_the_matrix():
    rng = np.random.default_rng(1)
    lens = [3, 4, 2, 5]
    merges = _random_merges(rng, 4)
    S = _random_S(rng, lens, density=1.0)
    got, nz = oracle.consistency(S, lens, merges, T=1, h=3.0, theta=0.0)
    for key in S:
        assert nz[key] == 0
        np.testing.assert_array_equal(got[key], S[key])


def test_identity_stays_identity_and_plain_average():
    k, n = 5, 4
    lens = [n] * k
    rng = np.random.default_rng(2)
    merges = _random_merges(rng, k)
    S = {(a, b): np.eye(n) for a in range(k) for b in range(a + 1, k)}
    got, nz = oracle.consistency(S, lens, merges, T=k, h=1.0, theta=0.0)
    for key in S:
        assert nz[key] == k - 2
        np.testing.assert_allclose(got[key], np.eye(n), atol=1e-15)
    # T = k, h = 1: the plain average over all k sequences (x, y with S_xx = I)
    S = _random_S(rng, lens, density=0.7)
    got, _ = oracle.consistency(S, lens, merges, T=k, h=1.0, theta=0.0)
    mat = lambda a, b: S[(a, b)] if a < b else S[(b, a)].T
    eye = np.eye(n)
    for x, y in S:
        full = sum((mat(x, z) if z != x else eye) @ (mat(z, y) if z != y else eye) for z in range(k)) / k
        np.testing.assert_allclose(got[(x, y)], full, rtol=1e-13)


def test_swap_transposes():
    """Relaxing (y, x) through the same z gives the transpose: written here by
    swapping the roles through transposed inputs."""
    rng = np.random.default_rng(4)
    k = 5
    lens = [int(v) for v in rng.integers(2, 5, k)]
    merges = _random_merges(rng, k)
    S = _random_S(rng, lens, density=0.6)
    got, _ = oracle.consistency(S, lens, merges, T=4, h=3.0, theta=0.0)
    # relabel sequences in reverse order: pair (x, y) becomes (k-1-y, k-1-x)
    perm = [k - 1 - i for i in range(k)]
    S2 = {}
    for (a, b), M in S.items():
        a2, b2 = perm[a], perm[b]
        S2[(min(a2, b2), max(a2, b2))] = M if a2 < b2 else M.T
    m2 = np.array([[perm[a] if a < k else a, perm[b] if b < k else b] for a, b in merges])
    got2, _ = oracle.consistency(S2, [lens[perm[i]] for i in range(k)], m2, T=4, h=3.0, theta=0.0)
    for (x, y), R in got.items():
        np.testing.assert_allclose(got2[(perm[y], perm[x])], R.T, rtol=1e-13, atol=1e-15)
