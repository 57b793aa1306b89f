"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 scaled form <= 1e-5 on every posterior and distance (the
stage's accuracy bar); FP64 plain form <= 1e-9.  Sparse patterns must match
wherever |P - theta| > 1e-5.  FP32 results must come from the FP32 kernel:
the tests assert that no pair was handed to the FP64 form unless stated.
"""
import numpy as np
import pytest

import synth
from gpu_util import (TOL_F32, TOL_F64, TOL_LOGZ32, TOL_LOGZ64, compare_pair, dense_of,
                      guard_report, host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp


DENSE = 1e-30     # threshold that keeps every non-negligible entry


def _run(qp, fam, prm, **kw):
    return qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, **kw)


def _no_fallback(res):
    assert res.n_fallback == 0, f"FP32 guards fired: {guard_report(res)} first event {res.guard_info}"


@pytest.mark.parametrize("precision,tol,tlz", [("f32", TOL_F32, TOL_LOGZ32), ("f64", TOL_F64, TOL_LOGZ64)])
def test_small_family_all_pairs_dense(qp, precision, tol, tlz):
    """8 sequences, lengths 100-150 (the small configuration), every pair, every cell."""
    fam = synth.make_family("c1", 1)
    prm = synth.default_params(threshold=DENSE)
    res = _run(qp, fam, prm, precision=precision)
    assert res.n_pairs == 28
    _no_fallback(res)
    worst = 0.0
    for p, (a, b) in enumerate(fam.pairs()):
        worst = max(worst, compare_pair(res, fam, p, a, b, prm, tol, tlz)["p_err"])
    print(f"{precision}: worst |dP| = {worst:.3e}")


@pytest.mark.parametrize("precision,tol,tlz", [("f32", TOL_F32, TOL_LOGZ32), ("f64", TOL_F64, TOL_LOGZ64)])
def test_small_family_threshold_pattern(qp, precision, tol, tlz):
    fam = synth.make_family("c1", 2)
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm, precision=precision)
    _no_fallback(res)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, tol, tlz, dense=False)


EDGE_LENGTHS = [1, 2, 3, 31, 32, 33, 95, 96, 97, 126, 127, 128, 129, 200, 255, 256, 257, 300]


@pytest.mark.parametrize("precision,tol,tlz", [("f32", TOL_F32, TOL_LOGZ32), ("f64", TOL_F64, TOL_LOGZ64)])
def test_edge_lengths(qp, precision, tol, tlz):
    """Lengths at lane, rows-per-lane and strip boundaries, m >> n and n >> m."""
    rng = np.random.Generator(np.random.PCG64(77))
    q = synth.background()
    root = rng.choice(20, size=320, p=q).astype(np.uint8)
    seqs = []
    for L in EDGE_LENGTHS:
        leaf = synth.evolve(rng, root[:L], 0.2, q)[:L]
        if leaf.size < L:
            leaf = np.concatenate([leaf, rng.choice(20, size=L - leaf.size, p=q).astype(np.uint8)])
        seqs.append("".join(synth.ALPHABET[c] for c in leaf))
    fam = synth.family_from_strings(seqs)
    prm = synth.default_params(threshold=DENSE)
    res = _run(qp, fam, prm, precision=precision)
    _no_fallback(res)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, tol, tlz)


@pytest.mark.parametrize("combine", ["mean", "hmm", "pf"])
def test_combination_modes(qp, combine):
    fam = synth.star_family(5, 5, (80, 180), 0.3)
    prm = synth.default_params(threshold=DENSE, combine=combine)
    res = _run(qp, fam, prm)
    _no_fallback(res)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32)


def test_nondefault_parameters(qp):
    """Non-uniform start, unequal end weights, other gap constants."""
    prm = synth.default_params(delta1=0.07, eps1=0.55, delta2=0.03, eps2=0.85,
                               gap_open=-5.0, gap_ext=-2.0, temperature=2.0, threshold=DENSE)
    prm = prm.replace(pi=np.array([0.6, 0.1, 0.15, 0.05, 0.1]),
                      end_w=np.array([1.0, 0.7, 0.4, 0.9, 0.2]))
    fam = synth.star_family(8, 5, (100, 260), 0.35)
    for precision, tol, tlz in (("f32", TOL_F32, TOL_LOGZ32), ("f64", TOL_F64, TOL_LOGZ64)):
        res = _run(qp, fam, prm, precision=precision)
        _no_fallback(res)
        for p, (a, b) in enumerate(fam.pairs()):
            compare_pair(res, fam, p, a, b, prm, tol, tlz)


def test_identical_and_unrelated_sequences(qp):
    """Range stress for the FP32 rescaling: identical sequences (totals grow by
    ~e^2.6 per residue) and unrelated random sequences."""
    rng = np.random.Generator(np.random.PCG64(3))
    q = synth.background()
    s = "".join(synth.ALPHABET[c] for c in rng.choice(20, size=400, p=q))
    r1 = "".join(synth.ALPHABET[c] for c in rng.choice(20, size=380, p=q))
    r2 = "".join(synth.ALPHABET[c] for c in rng.choice(20, size=350, p=q))
    fam = synth.family_from_strings([s, s, r1, r2])
    prm = synth.default_params(threshold=DENSE)
    res = _run(qp, fam, prm)
    _no_fallback(res)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32)


def test_swap_gives_transpose(qp):
    fam = synth.star_family(12, 2, (150, 220), 0.3)
    rev = synth.family_from_strings([fam.seq(1), fam.seq(0)])
    prm = synth.default_params(threshold=DENSE)
    r1 = _run(qp, fam, prm)
    r2 = _run(qp, rev, prm)
    m, n = fam.lengths
    D1 = dense_of(r1, 0, m, n)
    D2 = dense_of(r2, 0, n, m)
    assert np.abs(D2 - D1.T).max() <= 2 * TOL_F32
    assert abs(float(host(r1.dist64)[0, 1]) - float(host(r2.dist64)[0, 1])) <= 2 * TOL_F32


def test_pair_alone_equals_pair_in_batch(qp):
    """Batch invariance: a pair's FP32 result does not depend on what else is
    in the launch (bitwise)."""
    fam = synth.star_family(21, 10, (120, 300), 0.3)
    prm = synth.default_params(threshold=0.001)
    big = _run(qp, fam, prm)
    _no_fallback(big)
    a, b = 3, 7
    p = synth.pair_index(a, b, fam.k)
    alone = _run(qp, synth.family_from_strings([fam.seq(a), fam.seq(b)]), prm)
    m, n = fam.lengths[a], fam.lengths[b]
    assert np.array_equal(dense_of(big, p, m, n), dense_of(alone, 0, m, n))
    assert float(host(big.mea)[p]) == float(host(alone.mea)[0])
    assert float(host(big.log_z_hmm)[p]) == float(host(alone.log_z_hmm)[0])


def test_medium_family_sampled_pairs(qp):
    """64 sequences, lengths 200-400: the whole family in one launch (the
    benchmark's configuration); a seeded sample of pairs against the oracle."""
    fam = synth.make_family("c2", 1)
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    assert res.n_pairs == 2016
    _no_fallback(res)
    rng = np.random.Generator(np.random.PCG64(5))
    pl = list(fam.pairs())
    L = fam.lengths
    longest = max(range(len(pl)), key=lambda q: L[pl[q][0]] * L[pl[q][1]])
    shortest = min(range(len(pl)), key=lambda q: L[pl[q][0]] * L[pl[q][1]])
    sample = sorted(set(rng.choice(len(pl), size=24, replace=False).tolist() + [longest, shortest]))
    for q in sample:
        a, b = pl[q]
        compare_pair(res, fam, q, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)
    dist = host(res.dist)
    assert np.array_equal(dist, dist.T) and (np.diag(dist) == 0).all()
    assert (dist >= -1e-6).all() and (dist <= 1 + 1e-6).all()


def test_device_resident_input_and_output(qp):
    """Residues already on the device, results left on the device (torch views)."""
    import torch
    fam = synth.star_family(31, 6, (90, 140), 0.3)
    prm = synth.default_params(threshold=DENSE)
    dres = torch.from_numpy(fam.residues).cuda()
    r_dev = qp.qp_posteriors(dres, fam.offsets, prm, out_on_device=True, device=0)
    assert r_dev.on_device and r_dev.val.is_cuda
    r_host = _run(qp, fam, prm)
    assert r_dev.nnz == r_host.nnz
    assert np.array_equal(r_dev.val.cpu().numpy(), r_host.val)
    assert np.array_equal(r_dev.col.cpu().numpy(), r_host.col)


def test_invalid_residue_is_rejected(qp):
    fam = synth.family_from_strings(["ACDEFGHIK", "ACDXFGHIK"])
    with pytest.raises(qp.QpError) as e:
        _run(qp, fam, synth.default_params())
    assert e.value.code == 1


def test_longest_supported_sequence(qp):
    """The FP32 form's length limit on this device (every warp stages its
    pair's column residues in shared memory, in blocks of two warps): a
    family holding a sequence of exactly that length runs and matches the
    oracle, as columns (20 x L) and as rows (L x 30, hundreds of strips); one
    residue more is rejected with QP_EINVAL before anything runs."""
    lim = qp.qp_get_counter("f32_max_len")
    assert 10_000 < lim <= (1 << 20), lim
    rng = np.random.Generator(np.random.PCG64(2718))
    q = synth.background()
    long_seq = "".join(synth.ALPHABET[c] for c in rng.choice(20, size=lim, p=q))
    # the short sequences are copies of two stretches of the long one (one
    # letter changed), so each pair has an alignment band far into it
    a0, b0 = lim // 2, lim - 40
    s1 = long_seq[a0:a0 + 20]
    s1 = s1[:7] + ("A" if s1[7] != "A" else "C") + s1[8:]
    s2 = long_seq[b0:b0 + 30]
    fam = synth.family_from_strings([s1, long_seq, s2])
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    assert res.nnz > 0
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)
    res.free()
    over = synth.family_from_strings([s1, long_seq + "A", s2])
    with pytest.raises(qp.QpError) as e:
        _run(qp, over, prm)
    assert e.value.code == 1


def test_long_pairs_stay_in_fp32(qp):
    """Pairs of 500-700 residues (four to six strips): the per-lane exponents
    must follow the values down the strip chain, so no range guard fires."""
    fam = synth.star_family(44, 3, (560, 700), 0.3)
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    _no_fallback(res)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)


def _same_csr(a, b):
    for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val", "dist64", "mea",
                 "log_z_hmm", "log_z_pf", "pair_flags"):
        x, y = host(getattr(a, name)), host(getattr(b, name))
        assert np.array_equal(x, y), name


@pytest.mark.parametrize("which", ["edge", "long", "c1"])
def test_checkpointed_form_equals_stored(qp, which):
    """The checkpointed form recomputes each strip's backward values from the
    boundary row kept for it; the result must be bit-identical to the stored
    form (same start row, same instructions)."""
    if which == "c1":
        fam = synth.make_family("c1", 3)
    elif which == "long":
        fam = synth.star_family(45, 4, (560, 700), 0.3)
    else:
        rng = np.random.Generator(np.random.PCG64(78))
        q = synth.background()
        root = rng.choice(20, size=400, p=q).astype(np.uint8)
        seqs = []
        for L in (1, 33, 127, 128, 129, 255, 256, 257, 385):
            leaf = synth.evolve(rng, root[:L], 0.2, q)[:L]
            if leaf.size == 0:
                leaf = root[:1]
            seqs.append("".join(synth.ALPHABET[c] for c in leaf))
        fam = synth.family_from_strings(seqs)
    prm = synth.default_params(threshold=0.01)
    try:
        qp.qp_set_option("ckpt", 0)
        stored = _run(qp, fam, prm)
        qp.qp_set_option("ckpt", 1)
        ckpt = _run(qp, fam, prm)
    finally:
        qp.qp_set_option("ckpt", -1)
    _no_fallback(stored)
    _no_fallback(ckpt)
    _same_csr(stored, ckpt)
    if which == "long":
        for p, (a, b) in enumerate(fam.pairs()):
            compare_pair(ckpt, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)


def test_checkpointed_form_under_a_small_scratch_budget(qp):
    """A scratch budget too small for the stored form switches to the
    checkpointed form and cuts the grid; results stay the same."""
    fam = synth.make_family("c2", 2)
    prm = synth.default_params(threshold=0.01)
    ref = _run(qp, fam, prm)
    try:
        qp.qp_set_option("scratch_bytes", 256 << 20)
        small = _run(qp, fam, prm)
    finally:
        qp.qp_set_option("scratch_bytes", 0)
    _no_fallback(small)
    _same_csr(ref, small)


def test_long_family_sampled_pairs(qp):
    """100 sequences of 2000-4000 residues (three-domain roots, 4950 pairs) in
    one launch, in the form the library picks for them (checkpointed: the
    stored form would need ~130 MB per warp).  Seeded pairs against the
    oracle: totals, MEA score, distance and entry count for 12 pairs,
    posteriors for 2."""
    import concurrent.futures as cf
    import os
    import oracle
    fam = synth.make_family("c5", 1)
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    assert res.n_pairs == 4950
    _no_fallback(res)
    pl = list(fam.pairs())
    L = fam.lengths
    rng = np.random.Generator(np.random.PCG64(9))
    longest = max(range(len(pl)), key=lambda q: L[pl[q][0]] * L[pl[q][1]])
    sample = sorted(set(rng.choice(len(pl), size=11, replace=False).tolist() + [longest]))
    ref = oracle.pairs(fam, [pl[q] for q in sample], prm, threads=os.cpu_count())
    lzh, lzp = host(res.log_z_hmm), host(res.log_z_pf)
    mea, dist = host(res.mea), host(res.dist64)
    pno = host(res.pair_nnz_off)
    for i, q in enumerate(sample):
        a, b = pl[q]
        mn = min(L[a], L[b])
        assert abs(lzh[q] - ref["logz_hmm"][i]) <= TOL_LOGZ32 * abs(ref["logz_hmm"][i])
        assert abs(lzp[q] - ref["logz_pf"][i]) <= TOL_LOGZ32 * abs(ref["logz_pf"][i])
        assert abs(mea[q] - ref["mea"][i]) <= TOL_F32 * mn
        assert abs(dist[a, b] - ref["dist"][i]) <= TOL_F32
        nnz = int(pno[q + 1] - pno[q])
        assert abs(nnz - int(ref["nnz"][i])) <= 2 + nnz // 1000, (nnz, ref["nnz"][i])
    dense = [longest, sample[0]]
    with cf.ThreadPoolExecutor(len(dense)) as ex:
        refs = list(ex.map(lambda q: oracle.pair(fam.codes(pl[q][0]), fam.codes(pl[q][1]), prm), dense))
    for q, r in zip(dense, refs):
        a, b = pl[q]
        compare_pair(res, fam, q, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False, ref=r)


def test_large_family_sampled_pairs(qp):
    """500 sequences of 150-500 residues (124,750 pairs, random-tree family)
    in one launch; a seeded 0.5% sample of pairs (624) against the oracle:
    totals, MEA score, distance and entry count; posteriors for 4 pairs."""
    import os
    import oracle
    fam = synth.make_family("c3", 1)
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    assert res.n_pairs == 124750
    _no_fallback(res)
    pl = list(fam.pairs())
    L = fam.lengths
    rng = np.random.Generator(np.random.PCG64(11))
    sample = np.sort(rng.choice(len(pl), size=624, replace=False))
    ref = oracle.pairs(fam, [pl[q] for q in sample], prm, threads=os.cpu_count())
    lzh, lzp = host(res.log_z_hmm), host(res.log_z_pf)
    mea, dist = host(res.mea), host(res.dist64)
    pno = host(res.pair_nnz_off)
    a_s = np.array([pl[q][0] for q in sample])
    b_s = np.array([pl[q][1] for q in sample])
    mn = np.minimum(L[a_s], L[b_s])
    assert np.all(np.abs(lzh[sample] - ref["logz_hmm"]) <= TOL_LOGZ32 * np.abs(ref["logz_hmm"]))
    assert np.all(np.abs(lzp[sample] - ref["logz_pf"]) <= TOL_LOGZ32 * np.abs(ref["logz_pf"]))
    assert np.all(np.abs(mea[sample] - ref["mea"]) <= TOL_F32 * mn)
    assert np.abs(dist[a_s, b_s] - ref["dist"]).max() <= TOL_F32
    nnz = pno[sample + 1] - pno[sample]
    assert np.all(np.abs(nnz - ref["nnz"]) <= 2), np.abs(nnz - ref["nnz"]).max()
    d = host(res.dist)
    assert np.array_equal(d, d.T) and (np.diag(d) == 0).all()
    for q in sample[:4]:
        a, b = pl[q]
        compare_pair(res, fam, int(q), a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)


def test_millions_of_short_pairs(qp):
    """3000 sequences of 8-24 residues: 4.5 million pairs in one launch (far
    more work items than the C3 family's 124,750).  A seeded sample of 300
    pairs against the oracle (totals, MEA, distance, entry count), the
    distance matrix symmetric with a zero diagonal, and offsets that add up."""
    import os
    import oracle
    fam = synth.star_family(101, 3000, (12, 20), 0.3, keep=(8, 24))
    k = fam.k
    prm = synth.default_params(threshold=0.01)
    res = _run(qp, fam, prm)
    P = k * (k - 1) // 2
    assert res.n_pairs == P
    _no_fallback(res)
    L = np.asarray(fam.lengths)
    rng = np.random.Generator(np.random.PCG64(12))
    a_s = rng.integers(0, k - 1, size=300)
    b_s = np.array([int(rng.integers(a + 1, k)) for a in a_s])
    sample = a_s * k - a_s * (a_s + 1) // 2 + (b_s - a_s - 1)
    ref = oracle.pairs(fam, list(zip(a_s.tolist(), b_s.tolist())), prm, threads=os.cpu_count())
    lzh, lzp = host(res.log_z_hmm), host(res.log_z_pf)
    mea, dist = host(res.mea), host(res.dist64)
    pno, pro = host(res.pair_nnz_off), host(res.pair_row_off)
    mn = np.minimum(L[a_s], L[b_s])
    assert np.all(np.abs(lzh[sample] - ref["logz_hmm"]) <= TOL_LOGZ32 * np.abs(ref["logz_hmm"]))
    assert np.all(np.abs(lzp[sample] - ref["logz_pf"]) <= TOL_LOGZ32 * np.abs(ref["logz_pf"]))
    assert np.all(np.abs(mea[sample] - ref["mea"]) <= TOL_F32 * mn)
    assert np.abs(dist[a_s, b_s] - ref["dist"]).max() <= TOL_F32
    nnz = pno[sample + 1] - pno[sample]
    assert np.all(np.abs(nnz - ref["nnz"]) <= 2), np.abs(nnz - ref["nnz"]).max()
    d = host(res.dist)
    assert np.array_equal(d, d.T) and (np.diag(d) == 0).all()
    # rows: m + 1 per pair (a's length), entries: the last offset
    assert int(pro[-1]) == int(sum((L[a] + 1) * (k - 1 - a) for a in range(k)))
    assert int(pno[-1]) == int(res.nnz) and np.all(np.diff(pno) >= 0)
    for q in range(3):
        a, b = int(a_s[q]), int(b_s[q])
        compare_pair(res, fam, int(sample[q]), a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)


@pytest.mark.parametrize("wpp", [2])
@pytest.mark.parametrize("ckpt", [0, 1])
def test_warps_per_pair_equal_one(qp, wpp, ckpt):
    """Several warps sharing a pair (each taking every wpp-th strip and
    trailing its neighbour through the strip's boundary row) give the result
    of one warp per pair, bit for bit, in both forms."""
    # the c2 family fills the grid (every item on one warp of the two-warp
    # form); 44 sequences of 130-300 leave spare warps, so the longest items
    # are shared by two warps and the rest run alone in the same launch; the
    # small families share every item
    fams = [synth.make_family("c2", 3), synth.star_family(52, 44, (130, 300), 0.3),
            synth.star_family(46, 5, (560, 700), 0.3),
            synth.family_from_strings(["ACDEFGHIKLMNPQRSTVWY" * 7, "ACDEF", "WYVTSRQPNMLKIHGFEDCA" * 9])]
    prm = synth.default_params(threshold=0.01)
    try:
        qp.qp_set_option("ckpt", ckpt)
        for fam in fams:
            qp.qp_set_option("wpp", 1)
            one = _run(qp, fam, prm)
            qp.qp_set_option("wpp", wpp)
            many = _run(qp, fam, prm)
            _no_fallback(one)
            _no_fallback(many)
            _same_csr(one, many)
    finally:
        qp.qp_set_option("wpp", 0)
        qp.qp_set_option("ckpt", -1)


def test_long_pair_without_fp64_scratch(qp):
    """A scratch budget below one FP64 CTA's need (here 32 MiB against 36 MiB
    for length 1500) leaves the FP64 follow-up out; pairs that stay in FP32
    give the same result as with it."""
    fam = synth.star_family(47, 2, (1450, 1500), 0.3)
    prm = synth.default_params(threshold=0.01)
    ref = _run(qp, fam, prm)
    try:
        qp.qp_set_option("scratch_bytes", 32 << 20)
        small = _run(qp, fam, prm)
    finally:
        qp.qp_set_option("scratch_bytes", 0)
    _no_fallback(ref)
    _no_fallback(small)
    _same_csr(ref, small)


def test_null_stream_waits_for_the_default_stream(qp):
    """With params.stream NULL the call runs on the library's stream, which
    must first wait for the work queued on the legacy default stream: here
    the device residues are written there behind a 0.1 s spin."""
    import torch
    fam = synth.star_family(5, 8, (100, 150), 0.3)
    prm = synth.default_params()
    ref = _run(qp, fam, prm)
    src = torch.from_numpy(fam.residues).cuda()
    dst = torch.zeros_like(src)
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)
    dst.copy_(src)
    got = qp.qp_posteriors(dst, fam.offsets, qp.make_params(prm, device=0))
    assert np.array_equal(got.dist64, ref.dist64)
    assert np.array_equal(got.mea, ref.mea)


def test_entry_pool_overflow_reruns_the_call(qp):
    """A call whose entries overflow the entry pool must run again with a
    larger pool and give the result of a call that fitted: nothing after the
    posterior kernels may read the overflowed pool (with or without an entry
    budget)."""
    fam = synth.make_family("c1", 4)
    prm = synth.default_params(threshold=0.001)
    ref = _run(qp, fam, prm)
    ref_b = _run(qp, fam, prm, entry_budget=(ref.nnz // 3) * 8)
    try:
        for budget in (0, (ref.nnz // 3) * 8):
            base = ref if budget == 0 else ref_b
            qp.qp_set_option("pool_entries", 1000)
            before = qp.qp_get_counter("pool_retries")
            r = _run(qp, fam, prm, entry_budget=budget)
            assert qp.qp_get_counter("pool_retries") > before, "the pool did not overflow"
            assert r.nnz == base.nnz and r.threshold_used == base.threshold_used
            for name in ("row_ptr", "pair_nnz_off", "col", "val"):
                assert np.array_equal(host(r.array(name)), host(base.array(name))), name
            r.free()
    finally:
        qp.qp_set_option("pool_entries", 0)
    ref.free()
    ref_b.free()


def test_a_strip_wait_that_runs_out_goes_to_fp64(qp):
    """Two warps sharing a pair wait for each other's boundary rows with a
    bounded number of polls.  With the limit cut to one poll (a runtime
    option; the one-warp kernel the benchmark runs is untouched) the first
    wait of the second warp runs out before its neighbour has produced the
    rows it needs: the pair must be flagged (sync guard), recomputed by the
    FP64 form, and still match the oracle; a normal call on the same device
    afterwards must succeed in FP32."""
    fam = synth.star_family(48, 4, (300, 420), 0.3)     # 3-4 strips per pair
    prm = synth.default_params(threshold=DENSE)
    try:
        qp.qp_set_option("wpp", 2)
        qp.qp_set_option("spin_limit", 1)
        res = _run(qp, fam, prm)
    finally:
        qp.qp_set_option("spin_limit", 0)
        qp.qp_set_option("wpp", 0)
    flags = host(res.pair_flags)
    sync = (flags & (1 << 12)) != 0
    assert res.n_fallback > 0 and sync.any(), f"no wait ran out: flags {flags}"
    assert ((flags[sync] & 1) == 1).all(), "a pair whose wait ran out was not recomputed in FP64"
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(res, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32)
    res.free()
    again = _run(qp, fam, prm)
    _no_fallback(again)
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(again, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32)


@pytest.mark.parametrize("wpb,copies,wpp", [(2, 16, 1), (8, 16, 1), (8, 1, 1), (8, 16, 2), (4, 16, 2)])
def test_table_copies_and_block_shapes_are_bit_identical(qp, wpb, copies, wpp):
    """The bank-sliced emission table (16 copies), blocks of up to 8 warps and
    up to 4 groups of 2 warps per block change where values come from, never
    the values: the result equals the 2-warp-block, one-table, one-warp-per-pair
    launch bit for bit."""
    fams = [synth.make_family("c2", 3), synth.family_from_strings(["ACDEFGHIKLMNPQRSTVWY" * 7, "ACDEF",
                                                                   "WYVTSRQPNMLKIHGFEDCA" * 9])]
    prm = synth.default_params(threshold=0.01)
    try:
        for fam in fams:
            qp.qp_set_option("warps_per_block", 2)
            qp.qp_set_option("tab_copies", 1)
            qp.qp_set_option("wpp", 1)
            ref = _run(qp, fam, prm)
            qp.qp_set_option("warps_per_block", wpb)
            qp.qp_set_option("tab_copies", copies)
            qp.qp_set_option("wpp", wpp)
            got = _run(qp, fam, prm)
            _no_fallback(ref)
            _no_fallback(got)
            _same_csr(ref, got)
    finally:
        qp.qp_set_option("warps_per_block", 0)
        qp.qp_set_option("tab_copies", -1)
        qp.qp_set_option("wpp", 0)
