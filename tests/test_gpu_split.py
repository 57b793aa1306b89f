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
