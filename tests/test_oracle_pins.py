"""Pins of the FP64 oracle against things other than itself.

Each check is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong transition, a swapped index, a missing start/end weight) fails
at least one of them:
  * brute-force enumeration of every state path / alignment / matching of
    tiny pairs (totals, every posterior, gap posteriors, MEA);
  * forward total == backward total on larger pairs;
  * posterior identities: every residue is emitted exactly once;
  * closed forms for m = n = 1 and m = 1;
  * the ungapped limit and the zero-temperature limit (best alignment);
  * swapping the sequences transposes everything.
"""
import math
import zlib

import numpy as np
import pytest

import oracle
import synth
from bruteforce import (aligned_pairs, alignments, gotoh, hmm_brute,
                        mea_brute, pf_brute, pf_weight)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_seq(rng, n, prm=None):
    """n random residue codes of the parameters' alphabet (20 or 4 letters)."""
    a = 4 if prm is not None and prm.alphabet == "nucleotide" else 20
    return rng.integers(0, a, size=n).astype(np.uint8)


def _odd_params():
    """Asymmetric, non-default parameters: a non-uniform start, unequal end
    weights and different gap constants, so that every term is exercised."""
    p = synth.default_params(delta1=0.07, eps1=0.55, delta2=0.03, eps2=0.85,
                             gap_open=-5.0, gap_ext=-2.0, temperature=2.0)
    pi = np.array([0.6, 0.1, 0.15, 0.05, 0.1])
    return p.replace(pi=pi, end_w=np.array([1.0, 0.7, 0.4, 0.9, 0.2]))


def _odd_nucleotide_params():
    """Nucleotide mode (GTR-derived tables, 4 letters) with the same odd
    start, end and gap constants."""
    p = synth.nucleotide_params(delta1=0.07, eps1=0.55, delta2=0.03, eps2=0.85,
                                gap_open=-5.0, gap_ext=-2.0, temperature=2.0)
    pi = np.array([0.6, 0.1, 0.15, 0.05, 0.1])
    return p.replace(pi=pi, end_w=np.array([1.0, 0.7, 0.4, 0.9, 0.2]))


PARAMS = {"default": synth.default_params(), "odd": _odd_params(),
          "nucleotide": _odd_nucleotide_params()}
SHAPES = [(1, 1), (1, 3), (3, 1), (2, 2), (2, 4), (4, 3), (3, 5), (5, 5)]


@pytest.mark.parametrize("pname", sorted(PARAMS))
@pytest.mark.parametrize("shape", SHAPES)
def test_hmm_equals_bruteforce(pname, shape):
    prm = PARAMS[pname]
    rng = _rng(zlib.crc32(repr((pname, shape)).encode()))
    for _ in range(3):
        x, y = _rand_seq(rng, shape[0], prm), _rand_seq(rng, shape[1], prm)
        Z, PM, GX, GY = hmm_brute(x, y, prm)
        r = oracle.pair(x, y, prm)
        assert abs(r["logz_hmm"] - math.log(Z)) < 1e-11 * max(1.0, abs(math.log(Z)))
        np.testing.assert_allclose(r["P_hmm"], PM, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(r["gx_hmm"], GX, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(r["gy_hmm"], GY, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("pname", sorted(PARAMS))
@pytest.mark.parametrize("shape", SHAPES)
def test_pf_equals_bruteforce(pname, shape):
    prm = PARAMS[pname]
    rng = _rng(1000 + zlib.crc32(repr((pname, shape)).encode()))
    for _ in range(3):
        x, y = _rand_seq(rng, shape[0], prm), _rand_seq(rng, shape[1], prm)
        Z, PP, GX, GY = pf_brute(x, y, prm)
        r = oracle.pair(x, y, prm)
        assert abs(r["logz_pf"] - math.log(Z)) < 1e-11 * max(1.0, abs(math.log(Z)))
        np.testing.assert_allclose(r["P_pf"], PP, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(r["gx_pf"], GX, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(r["gy_pf"], GY, rtol=1e-11, atol=1e-13)


def test_hmm_and_pf_bruteforce_6x6():
    prm = PARAMS["odd"]
    rng = _rng(66)
    x, y = _rand_seq(rng, 6), _rand_seq(rng, 6)
    r = oracle.pair(x, y, prm)
    Z, PM, _, _ = hmm_brute(x, y, prm)
    np.testing.assert_allclose(r["P_hmm"], PM, rtol=1e-11, atol=1e-13)
    Zp, PP, _, _ = pf_brute(x, y, prm)
    np.testing.assert_allclose(r["P_pf"], PP, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("combine", ["rms", "mean", "hmm", "pf"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (4, 4), (5, 3), (4, 6)])
def test_mea_equals_bruteforce(combine, shape):
    prm = PARAMS["odd"].replace(combine=combine)
    rng = _rng(7 + shape[0] * 10 + shape[1])
    for _ in range(3):
        x, y = _rand_seq(rng, shape[0], prm), _rand_seq(rng, shape[1], prm)
        r = oracle.pair(x, y, prm)
        best = mea_brute(r["P"])
        assert abs(r["mea"] - best) < 1e-12
        assert abs(r["dist"] - (1.0 - best / min(shape))) < 1e-12


def test_combination_modes():
    rng = _rng(5)
    x, y = _rand_seq(rng, 30), _rand_seq(rng, 25)
    base = PARAMS["default"]
    r = {c: oracle.pair(x, y, base.replace(combine=c)) for c in ("rms", "mean", "hmm", "pf")}
    a, b = r["hmm"]["P_hmm"], r["hmm"]["P_pf"]
    assert np.array_equal(r["hmm"]["P"], a)
    assert np.array_equal(r["pf"]["P"], b)
    np.testing.assert_allclose(r["mean"]["P"], 0.5 * (a + b), rtol=0, atol=1e-15)
    rms = r["rms"]["P"]
    # a power mean of order 2 lies between the arithmetic mean and the max
    assert (rms >= 0.5 * (a + b) - 1e-15).all()
    assert (rms <= np.maximum(a, b) + 1e-15).all()
    assert (rms >= np.minimum(a, b) - 1e-15).all()
    # and equals sqrt of the mean of squares: check one cell per row by value
    i = np.arange(a.shape[0])
    j = np.argmax(rms, axis=1)
    np.testing.assert_allclose(rms[i, j] ** 2 * 2.0, a[i, j] ** 2 + b[i, j] ** 2, rtol=1e-13)


@pytest.mark.parametrize("pname", sorted(PARAMS))
@pytest.mark.parametrize("shape", [(30, 40), (97, 64), (150, 150)])
def test_forward_equals_backward(pname, shape):
    prm = PARAMS[pname]
    rng = _rng(shape[0] * 1000 + shape[1])
    x, y = _rand_seq(rng, shape[0], prm), _rand_seq(rng, shape[1], prm)
    r = oracle.pair(x, y, prm)
    assert abs(r["logz_hmm"] - r["logz_hmm_bwd"]) < 1e-10 * abs(r["logz_hmm"])
    assert abs(r["logz_pf"] - r["logz_pf_bwd"]) < 1e-10 * max(1.0, abs(r["logz_pf"]))


@pytest.mark.parametrize("pname", sorted(PARAMS))
def test_posterior_identities(pname):
    """Each residue is emitted exactly once: by M (paired with some y_j) or
    by a gap state; so the row sum of P_M plus the row's gap posterior is 1,
    and likewise for columns, for both models."""
    prm = PARAMS[pname]
    fam = synth.star_family(3, 2, (60, 80), 0.3, alphabet=prm.alphabet)
    x, y = fam.codes(0), fam.codes(1)
    r = oracle.pair(x, y, prm)
    np.testing.assert_allclose(r["P_hmm"].sum(1) + r["gx_hmm"], 1.0, atol=1e-11)
    np.testing.assert_allclose(r["P_hmm"].sum(0) + r["gy_hmm"], 1.0, atol=1e-11)
    np.testing.assert_allclose(r["P_pf"].sum(1) + r["gx_pf"], 1.0, atol=1e-11)
    np.testing.assert_allclose(r["P_pf"].sum(0) + r["gy_pf"], 1.0, atol=1e-11)
    P = r["P"]
    assert (P >= 0).all() and (P <= 1 + 1e-12).all()
    assert (P.sum(1) <= math.sqrt(2) + 1e-12).all()
    assert 0.0 <= r["dist"] <= 1.0


@pytest.mark.parametrize("pname", sorted(PARAMS))
def test_closed_form_one_by_one(pname):
    """m = n = 1: no X->Y move exists, so the only path is one match."""
    prm = PARAMS[pname]
    n_alpha = 4 if prm.alphabet == "nucleotide" else 20
    for a in range(0, n_alpha, 7 if n_alpha == 20 else 1):
        for b in range(0, n_alpha, 5 if n_alpha == 20 else 1):
            r = oracle.pair(np.array([a], np.uint8), np.array([b], np.uint8), prm)
            z = prm.pi[0] * prm.emit_pair[a, b] * prm.end_w[0]
            assert abs(r["logz_hmm"] - math.log(z)) < 1e-13
            assert abs(r["logz_pf"] - prm.score[a, b] / prm.temperature) < 1e-13
            assert abs(r["P_hmm"][0, 0] - 1.0) < 1e-14
            assert abs(r["P_pf"][0, 0] - 1.0) < 1e-14
            assert abs(r["mea"] - 1.0) < 1e-14 and abs(r["dist"]) < 1e-14


@pytest.mark.parametrize("pname", sorted(PARAMS))
@pytest.mark.parametrize("n", [2, 5, 17])
def test_closed_form_one_by_n(pname, n):
    """m = 1: x_1 must be matched to some y_j, with y-gap runs (one state
    kind per run) before and after; sum the n placements in closed form."""
    prm = PARAMS[pname]
    rng = _rng(n)
    x = _rand_seq(rng, 1, prm)
    y = _rand_seq(rng, n, prm)
    q, p = prm.emit_bg, prm.emit_pair
    d1, e1, d2, e2 = prm.delta1, prm.eps1, prm.delta2, prm.eps2
    pi, tau = prm.pi, prm.end_w

    def pre(a):   # weight of reaching M after a leading y-run of length a
        if a == 0:
            return pi[0]
        return pi[2] * e1 ** (a - 1) * (1 - e1) + pi[4] * e2 ** (a - 1) * (1 - e2)

    def post(b):  # weight of a trailing y-run of length b after M, with the end
        if b == 0:
            return tau[0]
        return d1 * e1 ** (b - 1) * tau[2] + d2 * e2 ** (b - 1) * tau[4]

    qy = np.prod(q[y])
    terms = np.array([pre(j) * p[x[0], y[j]] * post(n - 1 - j) * qy / q[y[j]] for j in range(n)])
    Z = terms.sum()
    r = oracle.pair(x, y, prm)
    assert abs(r["logz_hmm"] - math.log(Z)) < 1e-12 * abs(math.log(Z))
    np.testing.assert_allclose(r["P_hmm"][0], terms / Z, rtol=1e-11, atol=1e-15)
    # partition function: gap-run weights exp((go + (g-1) ge)/T)
    T, go, ge = prm.temperature, prm.gap_open, prm.gap_ext
    run = lambda g: 1.0 if g == 0 else math.exp((go + (g - 1) * ge) / T)
    w = np.array([run(j) * math.exp(prm.score[x[0], y[j]] / T) * run(n - 1 - j) for j in range(n)])
    assert abs(r["logz_pf"] - math.log(w.sum())) < 1e-12 * max(1, abs(math.log(w.sum())))
    np.testing.assert_allclose(r["P_pf"][0], w / w.sum(), rtol=1e-11, atol=1e-15)


def test_ungapped_limit():
    """delta -> 0 and gap open -> -inf: only the ungapped alignment of equal
    lengths survives, P is the identity and the MEA distance is 0."""
    prm = synth.default_params(delta1=0.0, delta2=0.0, gap_open=-1e6)
    prm = prm.replace(pi=np.array([1.0, 0, 0, 0, 0]))
    rng = _rng(11)
    for L in (1, 4, 23):
        x, y = _rand_seq(rng, L), _rand_seq(rng, L)
        r = oracle.pair(x, y, prm)
        np.testing.assert_allclose(r["P"], np.eye(L), atol=1e-14)
        assert abs(r["mea"] - L) < 1e-11 and abs(r["dist"]) < 1e-12
        ref = math.log(np.prod(prm.emit_pair[x, y]))
        assert abs(r["logz_hmm"] - ref) < 1e-12 * max(1, abs(ref))


def _unique_best(x, y, prm):
    scores = []
    for ops in alignments(len(x), len(y)):
        scores.append((math.log(pf_weight(ops, x, y, prm)) * prm.temperature, ops))
    scores.sort(key=lambda t: -t[0])
    return scores[0], scores[1][0]


def test_zero_temperature_limit_enumerated():
    """T -> 0: the partition function concentrates on the best alignment
    (found here by enumerating every alignment)."""
    rng = _rng(23)
    base = synth.default_params(gap_open=-6.0, gap_ext=-1.0)
    done = 0
    while done < 4:
        x, y = _rand_seq(rng, 5), _rand_seq(rng, 6)
        (best, ops), second = _unique_best(x, y, base)
        if best - second < 1.0:
            continue
        prm = base.replace(temperature=0.02)
        r = oracle.pair(x, y, prm)
        ind = np.zeros((5, 6))
        for i, j in aligned_pairs(ops):
            ind[i - 1, j - 1] = 1.0
        np.testing.assert_allclose(r["P_pf"], ind, atol=1e-15 + 1e-12)
        assert abs(r["logz_pf"] * prm.temperature - best) < 1e-6
        done += 1


def test_zero_temperature_limit_gotoh():
    """Same limit on larger pairs against a textbook affine (Gotoh)
    max-plus alignment with traceback."""
    fam = synth.star_family(9, 4, (14, 18), 0.25)
    base = synth.default_params(gap_open=-6.0, gap_ext=-1.0)
    for a, b in ((0, 1), (1, 2), (2, 3)):
        x, y = fam.codes(a), fam.codes(b)
        best, pairs = gotoh(x, y, base)
        r_lo = oracle.pair(x, y, base.replace(temperature=0.05))
        assert abs(r_lo["logz_pf"] * 0.05 - best) < 0.05 * math.log(50)
        ind = np.zeros((len(x), len(y)))
        for i, j in pairs:
            ind[i - 1, j - 1] = 1.0
        r = oracle.pair(x, y, base.replace(temperature=0.01))
        # a unique optimum with margin >= 1 leaves <= e^-100 weight elsewhere;
        # ties (margin 0) would split the mass, so check agreement with the
        # argmax path where it is confident
        conf = r["P_pf"] > 0.999
        assert conf.sum() > 0
        assert (ind[conf] == 1.0).all()


@pytest.mark.parametrize("pname", sorted(PARAMS))
def test_swap_transposes(pname):
    prm = PARAMS[pname]
    # the swap symmetry needs symmetric parameters (start and end too)
    prm = prm.replace(pi=np.array([prm.pi[0], prm.pi[1], prm.pi[1], prm.pi[3], prm.pi[3]]),
                      end_w=np.array([1.0, 0.5, 0.5, 0.25, 0.25]))
    fam = synth.star_family(5, 2, (40, 60), 0.35, alphabet=prm.alphabet)
    x, y = fam.codes(0), fam.codes(1)
    r1 = oracle.pair(x, y, prm)
    r2 = oracle.pair(y, x, prm)
    np.testing.assert_allclose(r2["P"], r1["P"].T, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r2["P_hmm"], r1["P_hmm"].T, rtol=1e-12, atol=1e-15)
    assert abs(r1["logz_hmm"] - r2["logz_hmm"]) < 1e-12 * abs(r1["logz_hmm"])
    assert abs(r1["logz_pf"] - r2["logz_pf"]) < 1e-12 * max(1, abs(r1["logz_pf"]))
    assert abs(r1["dist"] - r2["dist"]) < 1e-13


def test_thread_pool_matches_single_pair():
    fam = synth.star_family(2, 5, (20, 40), 0.3)
    prm = synth.default_params()
    pl = list(fam.pairs())
    res = oracle.pairs(fam, pl, prm, threads=3)
    for q, (a, b) in enumerate(pl):
        r = oracle.pair(fam.codes(a), fam.codes(b), prm)
        assert res["mea"][q] == r["mea"] and res["dist"][q] == r["dist"]
        assert res["logz_hmm"][q] == r["logz_hmm"] and res["logz_pf"][q] == r["logz_pf"]
        assert res["nnz"][q] == int((r["P"] >= prm.threshold).sum())


def test_sparsify_is_threshold():
    P = np.array([[0.5, 0.01, 0.0099999], [0.0, 1.0, 0.2]])
    rp, col, val = oracle.sparsify(P, 0.01)
    assert rp.tolist() == [0, 2, 4]
    assert col.tolist() == [0, 1, 1, 2]
    assert val.tolist() == [0.5, 0.01, 1.0, 0.2]


def test_nucleotide_encoding_and_tables():
    """Nucleotide mode: A, C, G, T map to 0..3 (U read as T, either case),
    protein letters are rejected; the GTR-derived emission table is a
    symmetric joint distribution whose marginals are the base frequencies."""
    assert oracle.encode("ACGTUacgtu", "nucleotide").tolist() == [0, 1, 2, 3, 3, 0, 1, 2, 3, 3]
    with pytest.raises(ValueError):
        oracle.encode("ACGTE", "nucleotide")
    prm = synth.nucleotide_params()
    J = prm.emit_pair[:4, :4]
    assert abs(J.sum() - 1.0) < 1e-14 and np.allclose(J, J.T, atol=1e-15)
    np.testing.assert_allclose(J.sum(axis=1), prm.emit_bg[:4], atol=1e-14)
    assert (prm.emit_pair[4:, :] == 0).all() and (prm.emit_pair[:, 4:] == 0).all()
    # transitions (A<->G, C<->T) score above transversions
    s = prm.score
    assert s[0, 2] > s[0, 1] and s[1, 3] > s[1, 2] and (np.diag(s)[:4] > 0).all()
