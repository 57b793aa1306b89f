"""Entry budget (paper, Methods, "Other algorithmic improvements": the
posterior matrices are fitted into a given amount of memory by keeping fewer
entries) on the GPU.

For each budget of N entries the result must
  1. fit: nnz <= N;
  2. be the unbudgeted result of the same call filtered at threshold_used
     (same rows, columns and values, bit for bit);
  3. use the smallest threshold that fits the values the call computed
     (a property of the result: one unit lower keeps more than N);
  4. agree with the oracle's threshold for the same family within the
     posterior tolerance: the (N+1)-th largest value is 1-Lipschitz in the
     values, so it moves by at most the largest value error (1e-5 for the
     FP32 form, 1e-9 for FP64), plus one unit in the last place.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL_F32, TOL_F64, host

pytestmark = pytest.mark.gpu

THETA = 0.01


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_07437_b300 as qp
    qp.lib()
    return qp


@pytest.fixture(scope="module")
def fam():
    return synth.star_family(23, 12, (120, 220), 0.35)


@pytest.fixture(scope="module")
def oracle_values(fam):
    """Every posterior entry >= THETA of every pair, from the oracle (FP64)."""
    prm = synth.default_params(threshold=THETA)
    vals = []
    for a, b in fam.pairs():
        P = oracle.pair(fam.codes(a), fam.codes(b), prm)["P"]
        vals.append(P[P >= THETA])
    return np.concatenate(vals)


def _csr(res, f64):
    """(pair_nnz_off, row_ptr, col, val) as host arrays, val in the compared precision."""
    n = int(res.nnz)
    val = host(res.array("val64"))[:n] if f64 else host(res.array("val"))[:n]
    return (host(res.array("pair_nnz_off")).copy(), host(res.array("row_ptr")).copy(),
            host(res.array("col"))[:n].copy(), np.asarray(val).copy())


def _filtered(full, t, pro):
    """The CSR `full` keeping entries >= t (row pointers per pair)."""
    pno, rp, col, val = full
    keep = val >= t
    out_rp = np.empty_like(rp)
    out_pno = np.zeros_like(pno)
    cols, vals = [], []
    for p in range(len(pno) - 1):
        r0, r1 = pro[p], pro[p + 1]
        base = pno[p]
        acc = 0
        for r in range(r0, r1):
            out_rp[r] = acc
            if r + 1 < r1:
                e0, e1 = base + rp[r], base + rp[r + 1]
                k = keep[e0:e1]
                cols.append(col[e0:e1][k])
                vals.append(val[e0:e1][k])
                acc += int(k.sum())
        out_pno[p + 1] = out_pno[p] + acc
    cat = lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dt)
    return out_pno, out_rp, cat(cols, col.dtype), cat(vals, val.dtype)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_budget_fits_filters_and_matches_oracle(qp, fam, oracle_values, precision):
    f64 = precision == "f64"
    dt = np.float64 if f64 else np.float32
    bpe = 16 if f64 else 8
    tol = (TOL_F64 if f64 else TOL_F32)
    prm = synth.default_params(threshold=THETA, precision=precision)
    full_res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    assert full_res.threshold_used == float(dt(THETA))
    pro = host(full_res.array("pair_row_off"))
    full = _csr(full_res, f64)
    nnz = int(full_res.nnz)
    vals = full[3]
    for n_keep in (nnz, nnz - 1, nnz // 2, nnz // 10, 17, 1):
        res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, entry_budget=n_keep * bpe)
        t = res.threshold_used
        assert res.nnz <= n_keep
        got = _csr(res, f64)
        exp = _filtered(full, dt(t), pro)
        for g, x, name in zip(got, exp, ("pair_nnz_off", "row_ptr", "col", "val")):
            assert np.array_equal(g, x), f"n_keep={n_keep}: {name} differs from the filtered full result"
        assert np.count_nonzero(vals >= dt(t)) <= n_keep
        if dt(t) > dt(THETA):
            assert np.count_nonzero(vals >= np.nextafter(dt(t), dt(0))) > n_keep, "not the smallest threshold"
        else:
            assert nnz <= n_keep
        t_ora = oracle.budget_threshold(oracle_values, THETA, n_keep, np.float64)
        slack = tol + 2 * float(np.spacing(dt(max(t, t_ora))))
        assert abs(t - t_ora) <= slack, f"n_keep={n_keep}: threshold {t!r} vs oracle {t_ora!r}"
        res.free()
    full_res.free()


def test_budget_edges(qp, fam):
    prm = synth.default_params(threshold=THETA)
    full = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0)
    nnz = int(full.nnz)
    vmax = float(host(full.array("val"))[:nnz].max())
    # room for everything: the same result, the threshold unchanged
    big = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, entry_budget=10 * nnz * 8)
    assert big.nnz == nnz and big.threshold_used == float(np.float32(THETA))
    assert np.array_equal(host(big.array("col"))[:nnz], host(full.array("col"))[:nnz])
    # room for no entry (a budget below one entry): nothing kept, the
    # threshold one unit above the largest value
    none = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, entry_budget=7)
    assert none.nnz == 0
    assert none.threshold_used == float(np.nextafter(np.float32(vmax), np.float32(1)))
    assert (host(none.array("row_ptr")) == 0).all()
    # distances and MEA scores do not depend on the budget
    assert np.array_equal(host(none.dist64), host(full.dist64))
    for r in (full, big, none):
        r.free()


def test_budget_on_device_and_graph_relaunch(qp, fam):
    """Device output through the captured call sequence, twice (the second
    call relaunches the graph), equals the host output."""
    import torch
    prm = synth.default_params(threshold=THETA)
    host_res = qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, entry_budget=4000 * 8)
    d_res = torch.from_numpy(fam.residues).cuda()
    before = qp.qp_get_counter("graph_relaunches")
    for _ in range(3):
        r = qp.qp_posteriors(d_res, fam.offsets, prm, device=0, out_on_device=True, entry_budget=4000 * 8)
        assert r.threshold_used == host_res.threshold_used and r.nnz == host_res.nnz
        n = int(r.nnz)
        assert np.array_equal(host(r.array("col"))[:n], host(host_res.array("col"))[:n])
        assert np.array_equal(host(r.array("val"))[:n], host(host_res.array("val"))[:n])
        assert np.array_equal(host(r.array("row_ptr")), host(host_res.array("row_ptr")))
        r.free()
    assert qp.qp_get_counter("graph_relaunches") > before
    host_res.free()


def test_budget_rejected_by_server_and_negative(qp):
    prm = synth.default_params()
    with pytest.raises(qp.QpError) as e:
        qp.Server(qp.make_params(prm, entry_budget=1 << 20), 1 << 30)
    assert e.value.code == 1
    fam = synth.star_family(2, 3, (30, 40), 0.3)
    with pytest.raises(qp.QpError) as e:
        qp.qp_posteriors(fam.residues, fam.offsets, prm, device=0, entry_budget=-1)
    assert e.value.code == 1
