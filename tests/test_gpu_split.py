"""One family split into pair ranges (qp_posteriors_range) on the GPU.

The ranges of an equal-work split (qp_split_pairs), each computed on its own
and assembled by the gather's layout code, must equal the single call's
result bit for bit: same kernels, same values, only the pair range differs.
"""
import numpy as np
import pytest

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


def _same(got, full):
    assert set(got) == set(full)
    for name in full:
        a, b = np.asarray(got[name]), np.asarray(full[name])
        assert a.dtype == b.dtype and a.shape == b.shape, name
        assert a.tobytes() == b.tobytes(), name


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_ranges_assemble_to_the_full_result(qp, precision):
    from paper_1512_07437_b300 import dist as qd
    fam = synth.star_family(23, 12, (90, 300), 0.3)
    prm = synth.default_params(threshold=0.01, precision=precision)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm, out_on_device=True)
    full = qd.result_chunk(res)
    res.free()
    for n in (2, 3, 7):
        b = qp.qp_split_pairs(fam.offsets, n)
        chunks = []
        for i in range(n):
            r = qp.qp_posteriors_range(fam.residues, fam.offsets, prm, int(b[i]), int(b[i + 1]),
                                       out_on_device=bool(i % 2))
            assert r.n_pairs == b[i + 1] - b[i]
            chunks.append(qd.result_chunk(r))
            r.free()
        _same(qd.assemble(chunks), full)


def test_single_pair_ranges(qp):
    """Every pair on its own: the finest split."""
    from paper_1512_07437_b300 import dist as qd
    fam = synth.star_family(29, 5, (40, 140), 0.3)
    prm = synth.default_params(threshold=0.01)
    res = qp.qp_posteriors(fam.residues, fam.offsets, prm)
    full = qd.result_chunk(res)
    res.free()
    chunks = []
    for p in range(fam.n_pairs):
        r = qp.qp_posteriors_range(fam.residues, fam.offsets, prm, p, p + 1)
        chunks.append(qd.result_chunk(r))
        r.free()
    _same(qd.assemble(chunks), full)


def test_range_rejects_bad_bounds(qp):
    fam = synth.star_family(29, 4, (40, 60), 0.3)
    prm = synth.default_params()
    for lo, hi in ((3, 3), (-1, 2), (0, 7), (5, 4)):
        with pytest.raises(qp.QpError) as e:
            qp.qp_posteriors_range(fam.residues, fam.offsets, prm, lo, hi)
        assert e.value.code == 1


RESULT_ARRAYS = ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val", "dist", "dist64", "mea",
                 "log_z_hmm", "log_z_pf", "pair_flags")


@pytest.mark.parametrize("chunks,which,on_device", [(2, "c2", False), (5, "c2", False), (3, "growing", False),
                                                     (4, "c2", True)])
def test_host_output_in_ranges_equals_one_piece(qp, chunks, which, on_device):
    """Host output of a large family is computed in pair ranges, the arrays of
    a finished range copied to host memory while the next range computes
    (option host_chunks).  The result must equal the one-piece call bit for
    bit.  The "growing" family (lengths rising along the pair order, every
    cell kept) makes the first range's entry estimate too small, so the host
    block is grown and copied over between ranges.  One case passes the
    residues already on the device (no upload starts a range)."""
    if which == "c2":
        fam = synth.make_family("c2", 5)
        prm = synth.default_params(threshold=0.01)
    else:
        rng = np.random.Generator(np.random.PCG64(91))
        q = synth.background()
        seqs = ["".join(synth.ALPHABET[c] for c in rng.choice(20, size=L, p=q)) for L in range(20, 260, 20)]
        fam = synth.family_from_strings(seqs)
        prm = synth.default_params(threshold=1e-30)
    res = fam.residues
    if on_device:
        import torch
        res = torch.from_numpy(fam.residues).cuda()
    try:
        qp.qp_set_option("host_chunks", 1)
        ref = qp.qp_posteriors(fam.residues, fam.offsets, prm, out_on_device=False)
        qp.qp_set_option("host_chunks", chunks)
        got = qp.qp_posteriors(res, fam.offsets, prm, out_on_device=False)
    finally:
        qp.qp_set_option("host_chunks", 0)
    assert (got.n_pairs, got.n_rows, got.nnz) == (ref.n_pairs, ref.n_rows, ref.nnz)
    for name in RESULT_ARRAYS:
        a, b = np.asarray(got.array(name)), np.asarray(ref.array(name))
        assert a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes(), name
    assert got.n_fallback == ref.n_fallback
    got.free()
    ref.free()
