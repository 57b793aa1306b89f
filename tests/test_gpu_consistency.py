"""Selective consistency (paper, Methods, stage III and "Selective
consistency") on the GPU against the oracle.

Parity: both sides relax their own dense posteriors (threshold 1e-30, so no
entry is near a threshold) over the same seeded guide tree.  The posteriors
differ by at most 1e-5 (FP32 form); a product term of row sums at most
sqrt(2) then moves by at most 2 sqrt(2) 1e-5, and so does the average of
terms: the relaxed values must agree within 4e-5, and the kept pattern
outside that band around the output threshold.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import host

pytestmark = pytest.mark.gpu

DENSE = 1e-30
TOL = 4e-5


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp


@pytest.fixture(scope="module")
def small(qp):
    """7 sequences of 30-70 residues, their dense posteriors on the GPU and
    in the oracle, and a seeded guide tree."""
    fam = synth.star_family(71, 7, (30, 70), 0.3)
    prm = synth.default_params(threshold=DENSE)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    S = {}
    for a, b in fam.pairs():
        S[(a, b)] = oracle.pair(fam.codes(a), fam.codes(b), prm)["P"]
    merges = synth.random_guide_tree(5, fam.k)
    return fam, res, S, merges


def _dense(res, k, lens):
    out = {}
    pro = host(res.array("pair_row_off"))
    pno = host(res.array("pair_nnz_off"))
    rp_all = host(res.array("row_ptr"))
    col = host(res.array("col"))
    val = host(res.array("val")).astype(np.float64)
    p = 0
    for a in range(k):
        for b in range(a + 1, k):
            rp = rp_all[pro[p]:pro[p + 1]]
            D = np.zeros((lens[a], lens[b]))
            base = int(pno[p])
            for i in range(lens[a]):
                c = col[base + rp[i]:base + rp[i + 1]]
                assert (np.diff(c) > 0).all(), "columns must ascend within a row"
                D[i, c] = val[base + rp[i]:base + rp[i + 1]]
            out[(a, b)] = D
            p += 1
    return out


@pytest.fixture
def forms(qp):
    """Restores the automatic choice of the relaxation's form after a test
    that forces one."""
    yield
    for name in ("cons_form", "cons_chunk_rows", "cons_min_unit", "cons_wait_polls", "cons_stall_test",
                 "cons_ctas_per_sm"):
        qp.qp_set_option(name, -1 if name == "cons_form" else 0, device=0)


@pytest.mark.parametrize("T,h,n_max", [(200, 3.0, 200), (3, 3.0, 200), (5, 1.0, 200), (4, 3.0, 2), (1, 3.0, 200)])
def test_relaxation_matches_oracle(qp, small, T, h, n_max):
    _check_against_oracle(qp, small, T, h, n_max)


@pytest.mark.parametrize("form,chunk_rows", [(1, 0), (1, 7), (1, 1), (0, 0)])
def test_each_form_matches_oracle(qp, small, forms, form, chunk_rows):
    """The staged form (whole pairs, chunks of 7 rows, single rows) and the
    row form, each against the oracle."""
    qp.qp_set_option("cons_form", form)
    qp.qp_set_option("cons_chunk_rows", chunk_rows)
    for T, h, n_max in ((200, 3.0, 200), (4, 3.0, 2)):
        _check_against_oracle(qp, small, T, h, n_max)
        assert qp.qp_get_counter("consistency_form") == form


def _check_against_oracle(qp, small, T, h, n_max):
    fam, res, S, merges = small
    lens = [int(v) for v in fam.lengths]
    theta = 0.01
    got = qp.qp_consistency(res, fam.offsets, merges, T=T, n_max=n_max, h=h, threshold=theta)
    exp, nz = oracle.consistency(S, lens, merges, T=T, h=h, n_max=n_max, theta=theta)
    # the oracle's threshold applied to its unthresholded relaxation, for the band
    raw, _ = oracle.consistency(S, lens, merges, T=T, h=h, n_max=n_max, theta=-1.0)
    G = _dense(got, fam.k, lens)
    worst = 0.0
    for key in exp:
        kept_ref = raw[key] >= theta
        kept_gpu = G[key] > 0
        band = np.abs(raw[key] - theta) <= TOL
        assert not ((kept_ref != kept_gpu) & ~band).any(), f"pair {key}: pattern differs outside the band"
        both = kept_ref & kept_gpu
        if both.any():
            worst = max(worst, float(np.abs(G[key][both] - raw[key][both]).max()))
    assert worst <= TOL, worst
    assert got.threshold_used == float(np.float32(theta))
    # distances and MEA scores are those of the posteriors
    assert np.array_equal(host(got.dist64), host(res.dist64))
    got.free()


def test_no_relaxation_keeps_the_posteriors(qp, small):
    """T = 0 selects no third sequence: S'_xy = (2 S_xy) / 2 = S_xy exactly,
    filtered at the threshold."""
    fam, res, S, merges = small
    lens = [int(v) for v in fam.lengths]
    got = qp.qp_consistency(res, fam.offsets, merges, T=0, threshold=0.02)
    G = _dense(got, fam.k, lens)
    R = _dense(res, fam.k, lens)
    for key in G:
        exp = np.where(R[key] >= np.float32(0.02), R[key], 0.0)
        assert np.array_equal(G[key], exp), key
    got.free()


def test_host_device_paths_and_determinism(qp):
    """Host and device posteriors, host and device merges, host and device
    output: bit-identical results; two runs are identical; merges produced by
    qp_guide_tree on the device chain straight in."""
    import torch
    fam = synth.star_family(72, 12, (60, 140), 0.35)
    prm = synth.default_params(threshold=0.01)
    d_res = torch.from_numpy(fam.residues).cuda()
    post_h = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    post_d = qp.qp_posteriors(d_res, fam.offsets, prm, device=0, out_on_device=True)
    merges_d, _ = qp.qp_guide_tree(post_d.dist64)
    merges_h = merges_d.cpu().numpy()
    runs = [
        qp.qp_consistency(post_h, fam.offsets, merges_h, T=6),
        qp.qp_consistency(post_d, fam.offsets, merges_d, T=6),
        qp.qp_consistency(post_d, fam.offsets, merges_h, T=6, out_on_device=True),
        qp.qp_consistency(post_h, fam.offsets, merges_h, T=6),
    ]
    ref = runs[0]
    n = int(ref.nnz)
    assert n > 0
    for r in runs[1:]:
        assert int(r.nnz) == n
        for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val"):
            assert np.array_equal(host(r.array(name)), host(ref.array(name))), name
    for r in runs + [post_h, post_d]:
        r.free()


def test_rejects_bad_input(qp, small):
    fam, res, S, merges = small
    bad = merges.copy()
    bad[1] = bad[0]                                   # a node joined twice
    with pytest.raises(qp.QpError) as e:
        qp.qp_consistency(res, fam.offsets, bad)
    assert e.value.code == 1
    off = fam.offsets.copy()
    off[2] += 1                                       # lengths that do not match the posteriors
    with pytest.raises(qp.QpError) as e:
        qp.qp_consistency(res, off, merges)
    assert e.value.code == 1
    with pytest.raises(qp.QpError) as e:
        qp.qp_consistency(res, fam.offsets, merges, h=0.5)
    assert e.value.code == 1


def _entries(res, k, lens):
    """{(a, b): (row * n + column keys, values)} of a result, ascending keys."""
    pro = host(res.array("pair_row_off"))
    pno = host(res.array("pair_nnz_off"))
    rp_all = host(res.array("row_ptr"))
    col = host(res.array("col")).astype(np.int64)
    val = host(res.array("val")).astype(np.float64)
    out, p = {}, 0
    for a in range(k):
        for b in range(a + 1, k):
            rp = rp_all[pro[p]:pro[p + 1]].astype(np.int64)
            rows = np.repeat(np.arange(lens[a], dtype=np.int64), np.diff(rp))
            sl = slice(int(pno[p]), int(pno[p]) + int(rp[-1]))
            out[(a, b)] = (rows * lens[b] + col[sl], val[sl])
            p += 1
    return out


def _compare_entries(A, B, theta, tol):
    worst = 0.0
    for key in A:
        ka, va = A[key]
        kb, vb = B[key]
        both, ia, ib = np.intersect1d(ka, kb, assume_unique=True, return_indices=True)
        if both.size:
            worst = max(worst, float(np.abs(va[ia] - vb[ib]).max()))
        only_a = np.setdiff1d(np.arange(ka.size), ia)
        only_b = np.setdiff1d(np.arange(kb.size), ib)
        assert (np.abs(va[only_a] - theta) <= tol).all(), f"pair {key}: pattern differs outside the band"
        assert (np.abs(vb[only_b] - theta) <= tol).all(), f"pair {key}: pattern differs outside the band"
    return worst


def test_forms_agree_beyond_the_stage_buffers(qp, forms):
    """Sequences of 700-1000 residues with posteriors kept down to 1e-3: some
    matrices hold more entries than a stage buffer, so the staged form reads
    those from global memory.  Staged (whole pairs and 50-row chunks) and row
    forms agree within 1e-6: both sum the same products in fixed point (units
    2^-30 and at most 2^-21), which differ by rounding alone; the multiply-add
    counts are equal."""
    import torch
    fam = synth.star_family(73, 9, (700, 1000), 0.35)
    prm = synth.default_params(threshold=1e-3)
    post = qp.qp_posteriors(torch.from_numpy(fam.residues).cuda(), fam.offsets, prm, device=0, out_on_device=True)
    pno = host(post.array("pair_nnz_off"))
    assert int(np.diff(pno).max()) > 4096 + 1536, "no matrix beyond the stage buffers"
    merges = synth.random_guide_tree(6, fam.k)
    lens = [int(v) for v in fam.lengths]
    got, fma = {}, {}
    for name, form, chunk in (("row", 0, 0), ("staged", 1, 0), ("chunked", 1, 50)):
        qp.qp_set_option("cons_form", form)
        qp.qp_set_option("cons_chunk_rows", chunk)
        r = qp.qp_consistency(post, fam.offsets, merges, T=200, threshold=2e-3, out_on_device=True)
        assert qp.qp_get_counter("consistency_form") == form
        fma[name] = qp.qp_get_counter("consistency_fma")
        got[name] = _entries(r, fam.k, lens)
        r.free()
    post.free()
    assert fma["row"] == fma["staged"] == fma["chunked"] > 0
    for name in ("staged", "chunked"):
        assert _compare_entries(got["row"], got[name], 2e-3, 1e-6) <= 1e-6, name


def test_forms_agree_on_long_sequences(qp, forms):
    """Sequences of 2000-2600 residues: one CTA's accumulator holds fewer
    than 16 rows of the longest, so the staged form takes stage buffers of
    an eighth of its shared memory and reads more z from global memory.  It
    agrees with the row form within 1e-6 (both sum the same products in
    fixed point) and counts the same multiply-adds."""
    import torch
    fam = synth.star_family(29, 6, (2000, 2600), 0.3)
    prm = synth.default_params(threshold=0.01)
    post = qp.qp_posteriors(torch.from_numpy(fam.residues).cuda(), fam.offsets, prm, device=0, out_on_device=True)
    merges = synth.random_guide_tree(3, fam.k)
    lens = [int(v) for v in fam.lengths]
    got, fma = {}, {}
    for name, form in (("row", 0), ("staged", 1)):
        qp.qp_set_option("cons_form", form)
        r = qp.qp_consistency(post, fam.offsets, merges, T=200, threshold=0.01, out_on_device=True)
        assert qp.qp_get_counter("consistency_form") == form
        fma[name] = qp.qp_get_counter("consistency_fma")
        got[name] = _entries(r, fam.k, lens)
        r.free()
    post.free()
    assert fma["row"] == fma["staged"] > 0
    assert _compare_entries(got["row"], got["staged"], 0.01, 1e-6) <= 1e-6


def test_staged_launch_shapes_are_bit_identical(qp, forms):
    """The staged form with one or two CTAs per SM (chunks of different
    heights) and with 3-row chunks gives the same result bit for bit: every
    sum is exact in the fixed-point unit, whatever the chunking, the order of
    the products, or which warp refills a stage buffer."""
    import torch
    fam = synth.star_family(41, 24, (150, 420), 0.35)
    prm = synth.default_params(threshold=0.01)
    post = qp.qp_posteriors(torch.from_numpy(fam.residues).cuda(), fam.offsets, prm, device=0, out_on_device=True)
    merges = synth.random_guide_tree(8, fam.k)
    got = {}
    for name, ctas, chunk in (("two", 2, 0), ("one", 1, 0), ("rows3", 2, 3)):
        qp.qp_set_option("cons_form", 1)
        qp.qp_set_option("cons_ctas_per_sm", ctas)
        qp.qp_set_option("cons_chunk_rows", chunk)
        r = qp.qp_consistency(post, fam.offsets, merges, T=200, threshold=0.01)
        assert qp.qp_get_counter("consistency_form") == 1
        got[name] = {a: host(r.array(a)).copy() for a in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val")}
        r.free()
    post.free()
    assert got["two"]["col"].size > 0
    for name in ("one", "rows3"):
        for a in got["two"]:
            assert np.array_equal(got["two"][a], got[name][a]), (name, a)


def test_staged_form_hands_a_coarse_unit_to_the_row_form(qp, small, forms):
    """When the bound on the sums would need a unit coarser than allowed, the
    call runs the row form: asking for 2^-31 forces that here, and the result
    is the row form's, bit for bit."""
    fam, res, S, merges = small
    lens = [int(v) for v in fam.lengths]
    qp.qp_set_option("cons_form", 0)
    ref = qp.qp_consistency(res, fam.offsets, merges, T=200)
    qp.qp_set_option("cons_form", 1)
    qp.qp_set_option("cons_min_unit", 31)
    got = qp.qp_consistency(res, fam.offsets, merges, T=200)
    assert qp.qp_get_counter("consistency_form") == 0
    for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val"):
        assert np.array_equal(host(got.array(name)), host(ref.array(name))), name
    got.free()
    ref.free()


@pytest.mark.parametrize("T", [200, 5])
def test_relaxation_at_c2_lengths_matches_oracle(qp, T):
    """Ten sequences of the 64-sequence benchmark family's lengths (200-400,
    star tree, 40% substitution), dense posteriors on both sides (threshold
    1e-30: no input entry near a threshold), a seeded guide tree; every pair
    relaxed against the oracle within 4e-5, patterns equal outside that band.
    With dense inputs every B is larger than a stage buffer (global reads),
    and each pair spans several row chunks."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    fam = synth.star_family(74, 10, (200, 400), 0.40, keep=(200, 400))
    prm = synth.default_params(threshold=DENSE)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    pl = list(fam.pairs())
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        S = dict(zip(pl, ex.map(lambda ab: oracle.pair(fam.codes(ab[0]), fam.codes(ab[1]), prm)["P"], pl)))
    merges = synth.random_guide_tree(9, fam.k)
    lens = [int(v) for v in fam.lengths]
    theta = 0.01
    got = qp.qp_consistency(res, fam.offsets, merges, T=T, threshold=theta)
    assert qp.qp_get_counter("consistency_form") == 1
    raw, nz = oracle.consistency(S, lens, merges, T=T, theta=-1.0)
    assert max(nz.values()) > 0
    G = _dense(got, fam.k, lens)
    worst = 0.0
    for key in raw:
        kept_ref = raw[key] >= theta
        kept_gpu = G[key] > 0
        band = np.abs(raw[key] - theta) <= TOL
        assert not ((kept_ref != kept_gpu) & ~band).any(), f"pair {key}: pattern differs outside the band"
        both = kept_ref & kept_gpu
        if both.any():
            worst = max(worst, float(np.abs(G[key][both] - raw[key][both]).max()))
    assert worst <= TOL, worst
    got.free()
    res.free()


@pytest.mark.parametrize("T", [200, 20])
def test_full_size_sampled_pairs(qp, T):
    """The 64-sequence benchmark family (200-400 residues, 2016 pairs) at the
    posterior threshold 0.01, in the launch configuration the benchmark
    times: three seeded pairs of the relaxed result against the oracle's
    relaxation of its own posteriors.

    An input entry within 2e-5 of the threshold may be kept on one side and
    dropped on the other (the posteriors agree to 1e-5).  The oracle bounds
    what such entries can add to each output cell, with B the matrices of
    those entries and S the oracle's kept entries:
        slack = (2 h_xy B_xy + sum_z (B_xz S_zy + S_xz B_zy + B_xz B_zy)) / (2 + |Z|),
    and the bar is 4e-5 + slack (cells kept on one side only must lie within
    that of the threshold)."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    import torch
    fam = synth.make_family("c2", 1)
    theta = 0.01
    prm = synth.default_params(threshold=theta)
    d_res = torch.from_numpy(fam.residues).cuda()
    post = qp.qp_posteriors(d_res, fam.offsets, prm, device=0, out_on_device=True)
    merges = synth.random_guide_tree(11, fam.k)
    got = qp.qp_consistency(post, fam.offsets, merges, T=T, threshold=theta, out_on_device=True)
    assert qp.qp_get_counter("consistency_form") == 1
    lens = [int(v) for v in fam.lengths]
    k = fam.k
    d = oracle.tree_distances(merges, k)
    rng = np.random.default_rng(17 + T)
    pl = list(fam.pairs())
    cand = [(x, y) for x, y in pl if any(z not in (x, y) and max(d[x, z], d[z, y]) <= T for z in range(k))]
    sample = [cand[i] for i in rng.permutation(len(cand))[:3]]
    need = set()
    for x, y in sample:
        need.add((x, y))
        for z in range(k):
            if z not in (x, y) and max(d[x, z], d[z, y]) <= T:
                need.update({(min(x, z), max(x, z)), (min(z, y), max(z, y))})
    need = sorted(need)
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        P = dict(zip(need, ex.map(lambda ab: oracle.pair(fam.codes(ab[0]), fam.codes(ab[1]), prm)["P"], need)))
    S = {ab: np.where(M >= theta, M, 0.0) for ab, M in P.items()}
    B = {ab: np.where(np.abs(M - theta) <= 2e-5, M, 0.0) for ab, M in P.items()}
    raw, nz = oracle.consistency(S, lens, merges, T=T, h=3.0, theta=-1.0, pairs=sample)

    def mat(M, a, b):
        return M[(a, b)] if a < b else M[(b, a)].T

    # the GPU's relaxed matrices of the sampled pairs (device result read back)
    pro = host(got.array("pair_row_off"))
    pno = host(got.array("pair_nnz_off"))
    rp_all = host(got.array("row_ptr"))
    col = host(got.array("col"))
    val = host(got.array("val")).astype(np.float64)
    for x, y in sample:
        p = x * k - x * (x + 1) // 2 + (y - x - 1)
        G = np.zeros((lens[x], lens[y]))
        rp = rp_all[pro[p]:pro[p + 1]]
        base = int(pno[p])
        for i in range(lens[x]):
            G[i, col[base + rp[i]:base + rp[i + 1]]] = val[base + rp[i]:base + rp[i + 1]]
        Z = [z for z in range(k) if z not in (x, y) and max(d[x, z], d[z, y]) <= T]
        assert len(Z) == nz[(x, y)] > 0
        hxy = 1.0 + 2.0 * min(len(Z), 200) / 200
        slack = 2.0 * hxy * B[(x, y)]
        for z in Z:
            slack = slack + mat(B, x, z) @ mat(S, z, y) + mat(S, x, z) @ mat(B, z, y) + mat(B, x, z) @ mat(B, z, y)
        slack = slack / (2.0 + len(Z))
        R = raw[(x, y)]
        bar = TOL + slack
        kept_ref, kept_gpu = R >= theta, G > 0
        assert not ((kept_ref != kept_gpu) & (np.abs(R - theta) > bar)).any(), f"pair {(x, y)}: pattern"
        both = kept_ref & kept_gpu
        assert (np.abs(G[both] - R[both]) <= bar[both]).all(), f"pair {(x, y)}: values"
    got.free()
    post.free()


def test_a_stage_wait_that_runs_out_fails_the_call_cleanly(qp, small, forms):
    """The staged form's waits on its stage buffers are bounded.  A test switch
    withholds the first batch's arrival, so no CTA's first wait can complete:
    each CTA gives up after the set number of waits, waits (bounded) for the
    copies it still has in flight and returns.  The call fails with QP_ECUDA
    and says why, and the next call on the same device gives the normal
    result."""
    fam, res, S, merges = small
    ref = qp.qp_consistency(res, fam.offsets, merges, T=200)
    qp.qp_set_option("cons_form", 1)
    qp.qp_set_option("cons_wait_polls", 64)
    qp.qp_set_option("cons_stall_test", 1)
    with pytest.raises(qp.QpError) as e:
        qp.qp_consistency(res, fam.offsets, merges, T=200)
    assert e.value.code == 3
    assert "did not complete" in str(e.value)
    qp.qp_set_option("cons_stall_test", 0)
    qp.qp_set_option("cons_wait_polls", 0)
    got = qp.qp_consistency(res, fam.offsets, merges, T=200)
    for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val"):
        assert np.array_equal(host(got.array(name)), host(ref.array(name))), name
    got.free()
    ref.free()
