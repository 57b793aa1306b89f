"""Serving loop with continuous batching (qp_server_* in include/qp.h).

Families submitted together share persistent launches; each family's result
must be what qp_posteriors gives for it alone, and the FP64 oracle checks a
sample of pairs.  Admission is by device memory, tested with a budget that
holds one family at a time."""
import re
import time
import zlib

import numpy as np
import pytest

import synth
from tests.gpu_util import TOL_F32, TOL_LOGZ32, compare_pair, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1512_07437_b300 as q
    q.lib()
    return q


def _mix():
    """Six families of different sizes and lengths (star and tree shaped)."""
    fams = []
    for i, (k, lr) in enumerate([(6, (60, 90)), (24, (120, 200)), (9, (250, 320)),
                                 (40, (50, 80)), (15, (180, 260)), (3, (400, 480))]):
        seed = zlib.crc32(f"server-mix-{i}".encode())
        if i % 2:
            fams.append(synth.tree_family(seed, k, lr, (0.05, 0.25), keep=lr, name=f"mix{i}"))
        else:
            fams.append(synth.star_family(seed, k, lr, 0.3))
    return fams


def _same_result(a, b, exact):
    """Compares two results of the same family (host arrays)."""
    for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col"):
        x, y = host(getattr(a, name)), host(getattr(b, name))
        assert np.array_equal(x, y), name
    for name, tol in (("val", TOL_F32), ("dist64", TOL_F32), ("mea", TOL_F32 * 500)):
        x, y = host(getattr(a, name)), host(getattr(b, name))
        assert x.shape == y.shape, name
        if exact:
            assert np.array_equal(x, y), name
        else:
            assert np.abs(x - y).max() <= tol, name
    for name in ("log_z_hmm", "log_z_pf"):
        x, y = host(getattr(a, name)), host(getattr(b, name))
        assert np.all(np.abs(x - y) <= TOL_LOGZ32 * np.maximum(1.0, np.abs(y))), name


def test_mix_equals_alone(qp):
    """Every family's result from the shared launches equals its result alone
    (bit for bit: the same kernel computes each pair independently), the
    launches really were shared, and sampled pairs match the FP64 oracle."""
    prm = synth.default_params()
    fams = _mix()
    alone = [qp.qp_posteriors(f.residues, f.offsets, prm) for f in fams]
    srv = qp.Server(prm, 64 << 30)
    try:
        tickets = [srv.submit(f.residues, f.offsets) for f in fams]
        got = [srv.poll(t, 120000) for t in tickets]
        st = srv.stats()
    finally:
        srv.destroy()
    assert all(g is not None for g in got)
    assert st["completed"] == len(fams) and st["failed"] == 0
    assert st["max_families_per_launch"] >= 2, st
    assert st["pairs_done"] == sum(f.k * (f.k - 1) // 2 for f in fams)
    for f, a, g in zip(fams, alone, got):
        assert g.k == f.k and g.nnz == a.nnz
        _same_result(g, a, exact=True)
    # oracle on a few pairs of three families
    import oracle
    for fi in (0, 2, 5):
        f, g = fams[fi], got[fi]
        for (a, b) in [(0, 1), (f.k - 2, f.k - 1)]:
            p = synth.pair_index(a, b, f.k)
            compare_pair(g, f, p, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)
    for r in alone + got:
        r.free()


def _needed_bytes(qp, prm, fam):
    """Device bytes the server asks for this family (from its refusal)."""
    srv = qp.Server(prm, 1)
    try:
        with pytest.raises(qp.QpError) as e:
            srv.submit(fam.residues, fam.offsets)
    finally:
        srv.destroy()
    assert e.value.code == 1
    m = re.search(r"needs (\d+) bytes \((\d+) resident \+ (\d+) kernel scratch\)", str(e.value))
    assert m, str(e.value)
    return int(m.group(2)), int(m.group(3))


def test_admission_by_memory(qp):
    """With a budget that holds one family, families run one at a time and
    all complete with the same result as alone."""
    prm = synth.default_params()
    fams = [synth.star_family(zlib.crc32(b"adm"), 12, (150, 200), 0.3)] * 4   # equal sizes
    res, scratch = _needed_bytes(qp, prm, fams[0])
    budget = scratch + res + res // 2
    alone = [qp.qp_posteriors(f.residues, f.offsets, prm) for f in fams]
    srv = qp.Server(prm, budget)
    try:
        tickets = [srv.submit(f.residues, f.offsets) for f in fams]
        got = [srv.poll(t, 120000) for t in tickets]
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["max_resident"] == 1, st
    assert st["completed"] == len(fams)
    for a, g in zip(alone, got):
        _same_result(g, a, exact=True)
        g.free()
        a.free()


def test_admission_two_at_a_time(qp):
    """A budget of two families lets the second be admitted while the first
    runs (it arrives while the first is on the GPU and shares its launches)."""
    prm = synth.default_params()
    fams = [synth.star_family(zlib.crc32(b"adm2"), 30, (200, 260), 0.3)] * 5
    res, scratch = _needed_bytes(qp, prm, fams[0])
    budget = scratch + 2 * res + res // 2
    srv = qp.Server(prm, budget)
    try:
        tickets = [srv.submit(f.residues, f.offsets) for f in fams]
        got = [srv.poll(t, 120000) for t in tickets]
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["max_resident"] == 2, st
    assert st["completed"] == len(fams)
    for f, g in zip(fams, got):
        d = host(g.dist64)
        assert d.shape == (f.k, f.k) and np.allclose(d, d.T) and (np.diag(d) == 0).all()
        g.free()


def test_staggered_arrivals(qp):
    """Families submitted while others are on the GPU join later launches
    and give the same results as alone."""
    prm = synth.default_params()
    fams = _mix()
    alone = [qp.qp_posteriors(f.residues, f.offsets, prm) for f in fams]
    srv = qp.Server(prm, 64 << 30)
    try:
        tickets = []
        for f in fams:
            tickets.append(srv.submit(f.residues, f.offsets))
            time.sleep(0.002)
        got = [srv.poll(t, 120000) for t in tickets]
    finally:
        srv.destroy()
    for a, g in zip(alone, got):
        _same_result(g, a, exact=True)
        a.free()
        g.free()


def test_device_resident_results(qp):
    prm = synth.default_params()
    f = _mix()[1]
    a = qp.qp_posteriors(f.residues, f.offsets, prm)
    srv = qp.Server(prm, 32 << 30, out_on_device=True)
    try:
        g = srv.poll(srv.submit(f.residues, f.offsets), 120000)
    finally:
        srv.destroy()
    assert g.on_device
    _same_result(g, a, exact=True)
    g.free()
    a.free()


def test_cancel_poll_and_errors(qp):
    prm = synth.default_params()
    big = synth.star_family(11, 200, (250, 300), 0.3)
    small = synth.star_family(12, 5, (50, 60), 0.3)
    srv = qp.Server(prm, 64 << 30)
    try:
        t_big = srv.submit(big.residues, big.offsets)
        assert srv.poll(t_big, 0) is None          # 19,900 pairs: still running
        t_c = srv.submit(small.residues, small.offsets)
        srv.cancel(t_c)
        with pytest.raises(qp.QpError) as e:
            srv.poll(t_c, 60000)
        assert e.value.code == 5
        t_s = srv.submit(small.residues, small.offsets)
        r = srv.poll(t_s, 120000)
        assert r is not None and r.n_pairs == 10
        r.free()
        r = srv.poll(t_big, 120000)
        assert r is not None and r.n_pairs == 200 * 199 // 2
        r.free()
        with pytest.raises(qp.QpError) as e:      # a ticket is consumed by its poll
            srv.poll(t_big, 0)
        assert e.value.code == 1
        bad = small.residues.copy()
        bad[3] = ord("B")
        with pytest.raises(qp.QpError) as e:
            srv.submit(bad, small.offsets)
        assert e.value.code == 1
        # a sequence longer than the FP32 form takes (the server's blocks of
        # four warps take less than qp_posteriors' two) is refused at submit
        too_long = synth.family_from_strings(["ACDEFGHIK", "A" * (qp.qp_get_counter("f32_max_len") + 1)])
        with pytest.raises(qp.QpError) as e:
            srv.submit(too_long.residues, too_long.offsets)
        assert e.value.code == 1
        st = srv.stats()
        assert st["cancelled"] == 1 and st["completed"] == 2 and st["resident"] == 0
    finally:
        srv.destroy()


def test_destroy_with_pending_work(qp):
    """Destroying a server with families queued and running returns after the
    device work ends; nothing is leaked into a second server."""
    prm = synth.default_params()
    fams = _mix()
    srv = qp.Server(prm, 64 << 30)
    for f in fams:
        srv.submit(f.residues, f.offsets)
    t0 = time.time()
    srv.destroy()
    assert time.time() - t0 < 60
    srv = qp.Server(prm, 64 << 30)
    try:
        r = srv.poll(srv.submit(fams[0].residues, fams[0].offsets), 60000)
        assert r is not None
        r.free()
    finally:
        srv.destroy()


def test_serving_trace_sampled_pairs(qp):
    """The first 12 families of the serving workload (Poisson arrivals,
    28-930 sequences, lengths 11-1000), submitted at their arrival times;
    one seeded pair per family against the oracle."""
    import os
    import oracle
    prm = synth.default_params(threshold=0.01)
    trace = synth.make_serving_trace(seed=4, n_families=12)
    srv = qp.Server(prm, 120 << 30)
    try:
        t0 = time.perf_counter()
        tickets = []
        for t_arr, f in trace:
            d = t0 + t_arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit(f.residues, f.offsets))
        got = [srv.poll(t, 300000) for t in tickets]
        st = srv.stats()
    finally:
        srv.destroy()
    assert st["completed"] == 12 and st["max_families_per_launch"] >= 2, st
    rng = np.random.Generator(np.random.PCG64(21))
    for (_, f), r in zip(trace, got):
        a, b = sorted(rng.choice(f.k, size=2, replace=False).tolist())
        p = synth.pair_index(a, b, f.k)
        ref = oracle.pairs(f, [(a, b)], prm, threads=1)
        assert abs(host(r.log_z_hmm)[p] - ref["logz_hmm"][0]) <= TOL_LOGZ32 * abs(ref["logz_hmm"][0])
        assert abs(host(r.log_z_pf)[p] - ref["logz_pf"][0]) <= TOL_LOGZ32 * abs(ref["logz_pf"][0])
        assert abs(host(r.dist64)[a, b] - ref["dist"][0]) <= TOL_F32
        pno = host(r.pair_nnz_off)
        assert abs(int(pno[p + 1] - pno[p]) - int(ref["nnz"][0])) <= 2
        r.free()


def test_fp64_follow_up_in_the_server(qp):
    """Pairs that the FP32 form hands to FP64 are recomputed by the server's
    FP64 follow-up launch.  Two warps per pair with the strip-wait limit cut
    to one poll (runtime testing knobs of the two-warp form) make waits run
    out; the flagged pairs must be recomputed in FP64 and match the oracle."""
    fam = synth.star_family(48, 4, (300, 420), 0.3)     # 3-4 strips per pair
    prm = synth.default_params(threshold=1e-4)
    try:
        qp.qp_set_option("wpp", 2)
        qp.qp_set_option("spin_limit", 1)
        srv = qp.Server(prm, 16 << 30)
        try:
            r = srv.poll(srv.submit(fam.residues, fam.offsets), 120000)
        finally:
            srv.destroy()
    finally:
        qp.qp_set_option("spin_limit", 0)
        qp.qp_set_option("wpp", 0)
    flags = host(r.pair_flags)
    sync = (flags & (1 << 12)) != 0
    assert r.n_fallback > 0 and sync.any(), f"no wait ran out: flags {flags}"
    assert ((flags[sync] & 1) == 1).all(), "a pair whose wait ran out was not recomputed in FP64"
    for p, (a, b) in enumerate(fam.pairs()):
        compare_pair(r, fam, p, a, b, prm, TOL_F32, TOL_LOGZ32, dense=False)
    r.free()
