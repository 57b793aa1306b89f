"""Guide tree (weighted UPGMA, paper Methods stage II) on the GPU vs the oracle.

Both sides compute in FP64 with the same join rule and tie rule, so merges
and heights must be bit-identical on the same input matrix.  Sizes the
oracle cannot finish (k above a few thousand, up to the k = 46340 limit) are
checked against an ultrametric built from gaps on a line, whose tree is known
in closed form: the gap of rank s is crossed at step s, at half its value,
joining the two clusters on either side of it.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp


FORMS = {"auto": (-1, 0), "cluster16": (2, 16), "cluster4": (2, 4), "smem": (1, 0), "global": (0, 0)}


@pytest.fixture(params=list(FORMS))
def form(qp, request):
    """The form of the kernel: automatic (the cluster form up to k of about
    660), the cluster form forced onto 16 or 4 CTAs, or one CTA with its
    per-slot state in shared or global memory -- each forced here at sizes
    the oracle finishes."""
    f, ctas = FORMS[request.param]
    qp.qp_set_option("tree_form", f)
    qp.qp_set_option("tree_ctas", ctas)
    yield request.param
    qp.qp_set_option("tree_form", -1)
    qp.qp_set_option("tree_ctas", 0)


def _fits_cluster(form, k):
    """Whether a forced cluster form holds k slots (rows of a slab x k x 8
    bytes within one CTA's shared memory)."""
    n = {"cluster16": 16, "cluster4": 4}.get(form)
    return n is None or -(-k // n) * (k + (k & 1)) * 8 + 16 * k < 220 * 1024


def _sym(rng, k, levels=None):
    A = rng.random((k, k)) if levels is None else rng.integers(0, levels, (k, k)) / levels
    D = np.triu(A, 1)
    return D + D.T


def _same(got, ref):
    merges, heights = got
    assert np.array_equal(np.asarray(merges), ref["merges"])
    assert np.array_equal(np.asarray(heights).view(np.int64), ref["heights"].view(np.int64)), \
        "heights differ in some bit"


def test_hand_example_and_tie_rule(qp):
    D = np.array([[0, 2, 4, 10], [2, 0, 6, 10], [4, 6, 0, 8], [10, 10, 8, 0]], dtype=float)
    m, h = qp.qp_guide_tree(D)
    assert m.tolist() == [[0, 1], [4, 2], [5, 3]] and h.tolist() == [1.0, 2.5, 4.5]
    m, h = qp.qp_guide_tree(np.ones((4, 4)) - np.eye(4))
    assert m.tolist() == [[0, 1], [4, 2], [5, 3]] and h.tolist() == [0.5, 0.5, 0.5]


@pytest.mark.parametrize("k", [2, 3, 31, 33, 64, 257, 700])
def test_random_matrix_bit_exact(qp, form, k):
    if not _fits_cluster(form, k):
        pytest.skip("the forced cluster form does not hold this k")
    D = _sym(np.random.default_rng(100 + k), k)
    _same(qp.qp_guide_tree(D), oracle.guide_tree(D))


@pytest.mark.parametrize("k,levels", [(300, 3), (129, 1), (500, 8)])
def test_ties_bit_exact(qp, form, k, levels):
    """Few distinct values: most steps choose among equal distances."""
    if not _fits_cluster(form, k):
        pytest.skip("the forced cluster form does not hold this k")
    D = _sym(np.random.default_rng(k * levels), k, levels)
    _same(qp.qp_guide_tree(D), oracle.guide_tree(D))


def test_only_upper_triangle_is_read(qp):
    rng = np.random.default_rng(5)
    D = _sym(rng, 90)
    L = D.copy()
    L[np.tril_indices(90, -1)] = rng.random(90 * 89 // 2) + 5.0
    np.fill_diagonal(L, -1.0)
    _same(qp.qp_guide_tree(L), oracle.guide_tree(D))


def test_device_input_equals_host_input(qp):
    import torch
    D = _sym(np.random.default_rng(9), 400)
    mh, hh = qp.qp_guide_tree(D)
    md, hd = qp.qp_guide_tree(torch.from_numpy(D).cuda())
    assert md.is_cuda and hd.is_cuda
    assert np.array_equal(md.cpu().numpy(), mh) and np.array_equal(hd.cpu().numpy(), hh)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ms, hs = qp.qp_guide_tree(torch.from_numpy(D).cuda())
    s.synchronize()
    assert np.array_equal(ms.cpu().numpy(), mh) and np.array_equal(hs.cpu().numpy(), hh)


def test_distances_of_the_posterior_stage(qp, form):
    """The matrix the posterior stage produces (dist64 of a 64-sequence
    family of 200-400 residues) in device memory, as the pipeline passes it."""
    fam = synth.star_family(41, 64, (200, 400), 0.4)
    res = qp.qp_posteriors(fam.residues, fam.offsets, synth.default_params(), out_on_device=True, device=0)
    d64 = res.dist64
    m, h = qp.qp_guide_tree(d64)
    ref = oracle.guide_tree(d64.cpu().numpy())
    res.free()
    _same((m.cpu().numpy(), h.cpu().numpy()), ref)


def _line_ultrametric_expected(pos, gap_of_rank_pos):
    """Merges of weighted UPGMA on the line ultrametric: step s crosses the
    gap of rank s at line position t, joining the clusters that hold the
    leaves at positions t - 1 and t.  A cluster sits in the smallest slot
    (leaf id) among its members, so the pair is ordered by that slot."""
    k = pos.size
    slot_at = np.empty(k, dtype=np.int64)
    slot_at[pos] = np.arange(k)
    parent = np.arange(k)
    root_id = np.arange(k)          # cluster id held by a root
    root_min = np.arange(k)         # smallest slot in the root's cluster

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    merges = np.empty((k - 1, 2), dtype=np.int32)
    for s, t in enumerate(gap_of_rank_pos):
        ra, rb = find(slot_at[t - 1]), find(slot_at[t])
        if root_min[ra] > root_min[rb]:
            ra, rb = rb, ra
        merges[s] = (root_id[ra], root_id[rb])
        parent[rb] = ra
        root_id[ra] = k + s
        root_min[ra] = min(root_min[ra], root_min[rb])
    return merges


def _device_line_ultrametric(k, seed):
    """D[p][q] = max of the gaps between the line positions of slots p and q,
    built on the device by a sparse table (range maxima), 1024 rows at a time.
    Gaps are a permutation of 1..k-1, so every average the tree takes is of
    equal values and exact."""
    import torch
    rng = np.random.default_rng(seed)
    pos = rng.permutation(k)                          # line position of slot p
    ranks = rng.permutation(k - 1)                    # gap t (t = 1..k-1) has value ranks[t-1] + 1
    gaps = np.zeros(k)
    gaps[1:] = ranks + 1.0
    g = torch.from_numpy(gaps).cuda()
    table = [g]
    while (1 << len(table)) <= k:
        prev, w = table[-1], 1 << (len(table) - 1)
        nxt = prev.clone()
        nxt[:k - w] = torch.maximum(prev[:k - w], prev[w:])
        table.append(nxt)
    st = torch.stack(table)                           # st[l][i] = max g[i .. i + 2^l - 1]
    P = torch.from_numpy(pos).cuda()
    D = torch.empty((k, k), dtype=torch.float64, device="cuda")
    for r0 in range(0, k, 1024):
        pi = P[r0:r0 + 1024, None]
        lo = torch.minimum(pi, P[None, :])
        hi = torch.maximum(pi, P[None, :])
        span = (hi - lo).clamp(min=1)
        lev = torch.floor(torch.log2(span.double())).long()
        # guard the floor of log2 against rounding at powers of two
        lev = torch.where((1 << (lev + 1)) <= span, lev + 1, lev)
        lev = torch.where((1 << lev) > span, lev - 1, lev)
        # both windows lie inside [lo + 1, hi] (the diagonal reads st[0][lo])
        first = torch.where(hi == lo, lo, lo + 1)
        v = torch.maximum(st[lev, first], st[lev, hi - (1 << lev) + 1])
        D[r0:r0 + 1024] = torch.where(hi == lo, torch.zeros_like(v), v)
        del pi, lo, hi, span, lev, v
    gap_pos_by_rank = np.argsort(ranks) + 1           # line position t of the gap of rank s
    return D, pos, gap_pos_by_rank


@pytest.mark.parametrize("k", [1100, 9000, 46340])
def test_line_ultrametric_any_size(qp, form, k):
    """Sizes the oracle cannot finish, up to the k limit (a 17 GB matrix):
    the closed-form tree of a line ultrametric, exactly.  k = 1100 is also
    checked against the oracle to tie the closed form to it."""
    import torch
    if form == "smem" and k > 8192:
        pytest.skip("above 8192 slots the state is always in global memory")
    if not _fits_cluster(form, k):
        pytest.skip("the forced cluster form does not hold this k")
    D, pos, gap_pos = _device_line_ultrametric(k, seed=k)
    m, h = qp.qp_guide_tree(D)
    m, h = m.cpu().numpy(), h.cpu().numpy()
    if k <= 1100:
        _same((m, h), oracle.guide_tree(D.cpu().numpy()))
    del D
    torch.cuda.empty_cache()
    assert np.array_equal(h, (np.arange(k - 1) + 1.0) * 0.5)
    assert np.array_equal(m, _line_ultrametric_expected(pos, gap_pos))
