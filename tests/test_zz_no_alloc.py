"""The allocation-free single-pair entry point (qp_pair_posteriors_static).

Some callers may not allocate device memory while they run (their memory
belongs to another allocator, or they cannot afford the synchronisation of
cudaMalloc/cudaFree).  This checks that the fixed-scratch entry point gives
the same pair results as qp_posteriors, on consecutive calls that reuse the
one scratch array, and that it refuses sizes beyond its fixed limit.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp, torch


def _static_call(qp, torch, x, y, prm, cap=None):
    m, n = len(x), len(y)
    res = torch.from_numpy(np.frombuffer((x + y).encode(), dtype=np.uint8).copy()).cuda()
    cap = m * n if cap is None else cap
    row_ptr = torch.full((m + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    val = torch.full((max(cap, 1),), -7.0, dtype=torch.float32, device="cuda")
    out = torch.full((4,), -7.0, dtype=torch.float64, device="cuda")
    nnz = qp.qp_pair_posteriors_static(res, m, n, prm, row_ptr, col, val, out)
    return (nnz, row_ptr.cpu().numpy(), col.cpu().numpy()[:nnz], val.cpu().numpy()[:nnz],
            out.cpu().numpy())


def _check_against_qp_posteriors(qp, x, y, prm, nnz, rp, col, val, out):
    """Both entry points run the same FP32 kernel on the same inputs, so every
    output must be identical, bit for bit."""
    fam = synth.family_from_strings([x, y])
    ref = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    rrp, rcol, rval, _ = ref.pair_csr(0)
    assert nnz == ref.nnz
    assert np.array_equal(rp, rrp)
    assert np.array_equal(col, rcol)
    assert np.array_equal(val.view(np.uint32), rval.view(np.uint32))
    expect = np.array([float(host(ref.mea)[0]), float(host(ref.dist64)[0, 1]),
                       float(host(ref.log_z_hmm)[0]), float(host(ref.log_z_pf)[0])])
    assert np.array_equal(out.view(np.uint64), expect.view(np.uint64)), (out, expect)
    ref.free()


def test_static_entry_matches_qp_posteriors_twice(env):
    qp, torch = env
    fam = synth.star_family(41, 4, (180, 300), 0.3)
    prm = synth.default_params(threshold=0.01)
    # two calls in a row with different shapes: the second must not see
    # anything left in the shared scratch by the first
    pairs = [(fam.seq(0), fam.seq(1)), (fam.seq(3)[:90], fam.seq(2))]
    for x, y in pairs:
        _check_against_qp_posteriors(qp, x, y, prm, *_static_call(qp, torch, x, y, prm))
    # and the first pair again, after the second
    _check_against_qp_posteriors(qp, *pairs[0], prm, *_static_call(qp, torch, *pairs[0], prm))


def test_static_entry_at_its_size_limit(env):
    qp, torch = env
    limit = qp.qp.QP_STATIC_MAX_LEN
    rng = np.random.Generator(np.random.PCG64(9))
    q = synth.background()
    root = rng.choice(20, size=limit, p=q).astype(np.uint8)
    x = "".join(synth.ALPHABET[c] for c in root)
    y = "".join(synth.ALPHABET[c] for c in synth.evolve(rng, root, 0.3, q)[:limit])
    prm = synth.default_params(threshold=1e-30)
    for _ in range(2):
        _check_against_qp_posteriors(qp, x, y, prm, *_static_call(qp, torch, x, y, prm))


def test_static_entry_rejects_what_it_cannot_hold(env):
    qp, torch = env
    limit = qp.qp.QP_STATIC_MAX_LEN
    prm = synth.default_params()
    with pytest.raises(qp.QpError) as e:
        _static_call(qp, torch, "A" * (limit + 1), "ACDE", prm)
    assert e.value.code == 1 and str(limit) in str(e.value)
    # an output capacity that is too small is reported with the needed count
    x, y = "ACDEFGHIKLMNPQRSTVWY" * 5, "ACDEFGHIKLMNPQRSTVWY" * 4
    with pytest.raises(qp.QpError) as e:
        _static_call(qp, torch, x, y, synth.default_params(threshold=1e-30), cap=3)
    assert e.value.code == 1 and "too small" in str(e.value)
