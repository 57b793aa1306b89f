"""Nucleotide mode (paper, Methods, "Other algorithmic improvements": a
nucleotide mode with a HOXD-style substitution matrix and a GTR model) on the
GPU against the FP64 oracle.

The kernels are the protein ones with 4-letter tables (GTR-derived, see
synth.nucleotide_params), so the bar is the same: every posterior and
distance within 1e-5 (FP32 form) or 1e-9 (FP64 form) of the oracle, sparse
patterns equal outside the guard band around the threshold.
"""
import numpy as np
import pytest

import synth
from gpu_util import (TOL_F32, TOL_F64, TOL_LOGZ32, TOL_LOGZ64, compare_pair, dense_of,
                      guard_report, host)

pytestmark = pytest.mark.gpu

DENSE = 1e-30


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp


def _nfam(seed, k, lens, s=0.3):
    return synth.star_family(seed, k, lens, s, alphabet="nucleotide")


@pytest.mark.parametrize("precision,tol,tlz", [("f32", TOL_F32, TOL_LOGZ32), ("f64", TOL_F64, TOL_LOGZ64)])
def test_all_pairs_dense(qp, precision, tol, tlz):
    """8 sequences of 150-400 nt (several 128-row strips and ragged tails):
    every pair, every cell."""
    fam = _nfam(31, 8, (150, 400))
    prm = synth.nucleotide_params(threshold=DENSE)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, precision=precision)
    assert res.n_fallback == 0, guard_report(res)
    worst = 0.0
    for p, (a, b) in enumerate(fam.pairs()):
        worst = max(worst, compare_pair(res, fam, p, a, b, prm, tol, tlz)["p_err"])
    print(f"nucleotide {precision}: worst |dP| = {worst:.3e}")
    res.free()


def test_medium_family_sampled_pairs(qp):
    """64 sequences of 400-800 nt at threshold 0.01, sampled pairs against the
    oracle (sparse pattern and values)."""
    fam = _nfam(32, 64, (400, 800), s=0.35)
    prm = synth.nucleotide_params(threshold=0.01)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    assert res.n_fallback == 0, guard_report(res)
    rng = np.random.default_rng(5)
    pl = list(fam.pairs())
    for idx in rng.choice(len(pl), 12, replace=False):
        a, b = pl[int(idx)]
        compare_pair(res, fam, int(idx), a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)
    res.free()


def test_letters(qp):
    """Lower case and U (read as T) give the same result; a protein letter is
    rejected in nucleotide mode and a nucleotide-only letter (U) in protein
    mode."""
    prm = synth.nucleotide_params(threshold=DENSE)
    x, y = "ACGTTGCAACGGTAC" * 7, "ACGTAGCATCGGTTCA" * 6
    ref = qp.qp_posteriors(*_pack([x, y]), prm, device=0)
    alt = qp.qp_posteriors(*_pack([x.lower(), y.replace("T", "U")]), prm, device=0)
    assert np.array_equal(host(alt.dist64), host(ref.dist64))
    assert np.array_equal(host(alt.array("val"))[:alt.nnz], host(ref.array("val"))[:ref.nnz])
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(*_pack([x, "ACGTEACGT"]), prm, device=0)
    assert e.value.code == 1 and "nucleotide" in str(e.value)
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(*_pack(["ACDU", "ACDE"]), synth.default_params(), device=0)
    assert e.value.code == 1
    ref.free()
    alt.free()


def _pack(seqs):
    fam = synth.family_from_strings(seqs, alphabet="nucleotide")
    return fam.residues, fam.offsets


def test_server_and_static_call(qp):
    """A server built on nucleotide parameters and the allocation-free call
    give the results of qp_posteriors bit for bit."""
    import torch
    prm = synth.nucleotide_params()
    fams = [_nfam(40 + i, k, (100, 300)) for i, k in enumerate((5, 9, 3))]
    alone = [qp.qp_posteriors(f.residues, f.offsets, prm, device=0) for f in fams]
    srv = qp.Server(prm, 8 << 30)
    try:
        got = [srv.poll(srv.submit(f.residues, f.offsets), 120000) for f in fams]
        with pytest.raises(qp.QpError):
            srv.submit(*_pack(["ACGT", "ACGE"]))
    finally:
        srv.destroy()
    for f, a, g in zip(fams, alone, got):
        assert g is not None and g.nnz == a.nnz
        assert np.array_equal(host(g.dist64), host(a.dist64))
        assert np.array_equal(host(g.array("col"))[:g.nnz], host(a.array("col"))[:a.nnz])
        assert np.array_equal(host(g.array("val"))[:g.nnz], host(a.array("val"))[:a.nnz])
    # the allocation-free single-pair call on the first pair of the first family
    f = fams[0]
    x, y = f.seq(0), f.seq(1)
    m, n = len(x), len(y)
    res = torch.from_numpy(np.frombuffer((x + y).encode(), dtype=np.uint8).copy()).cuda()
    row_ptr = torch.zeros(m + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(m * n, dtype=torch.int32, device="cuda")
    val = torch.zeros(m * n, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    nnz = qp.qp_pair_posteriors_static(res, m, n, prm, row_ptr, col, val, out)
    ref = alone[0]
    D = np.zeros((m, n))
    rp, c, v = row_ptr.cpu().numpy(), col.cpu().numpy()[:nnz], val.cpu().numpy()[:nnz]
    for i in range(m):
        D[i, c[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert nnz == int(host(ref.array("pair_nnz_off"))[1])
    assert np.abs(D - dense_of(ref, 0, m, n)).max() <= TOL_F32
    assert abs(out.cpu().numpy()[1] - float(host(ref.dist64)[0, 1])) <= TOL_F32
    for r in alone + got:
        r.free()
