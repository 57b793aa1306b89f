"""Multi-GPU host logic on CPU: world_size-2 gloo process group.

The posterior stage shards without any data-path exchange; ranks only agree
on timing.  These tests run the helpers bench.py uses for N > 1 in two
processes (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1512_07437_b300 import dist as qd
    try:
        assert qd.env() == (rank, world, rank)
        assert qd.init("gloo")
        qd.barrier()
        mx = qd.max_over_ranks(1.5 + rank)
        sm = qd.sum_over_ranks(1.0 + rank)
        # rank r processed (r + 1) * 1e6 units in (r + 1) * 0.5 s
        rate = qd.whole_job_rate((rank + 1) * 1e6, (rank + 1) * 0.5)
        seed = qd.rank_seed(1, rank)
        qd.barrier()
        qd.finalize()
        q.put((rank, mx, sm, rate, seed, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, None, repr(e)))


def test_two_rank_timing_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, mx, sm, rate, seed, err in out:
        assert err is None, err
        assert mx == 2.5 and sm == 3.0
        # all units (3e6) over the slowest rank's time (1.0 s)
        assert rate == pytest.approx(3e6)
    assert out[0][4] != out[1][4], "each rank draws its own workload"


def test_single_process_is_identity():
    from paper_1512_07437_b300 import dist as qd
    assert not qd.init("gloo")
    assert qd.max_over_ranks(2.0) == 2.0 and qd.sum_over_ranks(3.0) == 3.0
    assert qd.whole_job_rate(10.0, 2.0) == 5.0


# ---------------------------------------------------------------- one family split over ranks
def _synthetic_result(lens, seed):
    """A made-up single-rank result layout (random sparse matrices, values and
    distances) for a family with these lengths: the gather must rebuild it
    exactly from per-range chunks."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    k = len(lens)
    pro, pno, rps, cols, vals = [0], [0], [], [], []
    P = k * (k - 1) // 2
    dist = np.zeros((k, k), np.float32)
    d64 = np.zeros((k, k))
    for a in range(k):
        for b in range(a + 1, k):
            m, n = int(lens[a]), int(lens[b])
            cnt = rng.integers(0, min(4, n) + 1, m)
            rp = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
            rps.append(rp)
            for i in range(m):
                cols.append(np.sort(rng.choice(n, size=int(cnt[i]), replace=False)).astype(np.int32))
            vals.append(rng.random(int(rp[-1])).astype(np.float32))
            pro.append(pro[-1] + m + 1)
            pno.append(pno[-1] + int(rp[-1]))
            d = rng.random()
            dist[a, b] = dist[b, a] = np.float32(d)
            d64[a, b] = d64[b, a] = d
    return {"pair_row_off": np.array(pro, np.int64), "row_ptr": np.concatenate(rps),
            "pair_nnz_off": np.array(pno, np.int64), "col": np.concatenate(cols), "val": np.concatenate(vals),
            "dist": dist, "dist64": d64, "mea": rng.random(P), "log_z_hmm": rng.normal(size=P),
            "log_z_pf": rng.normal(size=P), "pair_flags": rng.integers(0, 8, P).astype(np.int32)}


def _chunk_of(full, lens, p0, p1):
    """What the range call documents for pairs p0 <= p < p1: chunk-relative
    offsets, the range's rows and entries, and distance matrices holding only
    the range's pairs."""
    import numpy as np
    pro, pno = full["pair_row_off"], full["pair_nnz_off"]
    c = {"pair_row_off": pro[p0:p1 + 1] - pro[p0], "row_ptr": full["row_ptr"][pro[p0]:pro[p1]],
         "pair_nnz_off": pno[p0:p1 + 1] - pno[p0], "col": full["col"][pno[p0]:pno[p1]],
         "val": full["val"][pno[p0]:pno[p1]]}
    for name in ("mea", "log_z_hmm", "log_z_pf", "pair_flags"):
        c[name] = full[name][p0:p1]
    k = len(lens)
    c["dist"] = np.zeros_like(full["dist"])
    c["dist64"] = np.zeros_like(full["dist64"])
    p = 0
    for a in range(k):
        for b in range(a + 1, k):
            if p0 <= p < p1:
                for name in ("dist", "dist64"):
                    c[name][a, b] = full[name][a, b]
                    c[name][b, a] = full[name][b, a]
            p += 1
    return c


def _same_layout(got, full):
    import numpy as np
    assert set(got) == set(full)
    for name in full:
        a, b = np.asarray(got[name]), np.asarray(full[name])
        assert a.dtype == b.dtype and a.shape == b.shape, name
        assert a.tobytes() == b.tobytes(), name


LENS = [37, 5, 61, 12, 44, 9, 30, 52, 18]


def _split_worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    from paper_1512_07437_b300 import dist as qd
    try:
        assert qd.init("gloo")
        off = np.concatenate([[0], np.cumsum(LENS)]).astype(np.int64)
        bounds = qd.split_bounds(off, world)
        full = _synthetic_result(LENS, seed=5)
        got = qd.gather_chunks(_chunk_of(full, LENS, int(bounds[rank]), int(bounds[rank + 1])))
        if rank == 0:
            _same_layout(got, full)
        else:
            assert got is None
        qd.finalize()
        q.put((rank, bounds.tolist(), None))
    except Exception as e:  # reported to the parent
        import traceback
        q.put((rank, None, traceback.format_exc()))


def test_two_ranks_gather_the_single_rank_layout():
    """Each of two gloo ranks holds the chunk of its equal-work pair range;
    the gather on rank 0 equals the single-rank layout bit for bit."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, bounds, err in out:
        assert err is None, err
    assert out[0][1] == out[1][1], "both ranks must agree on the split"


def _work(lens):
    import numpy as np
    k = len(lens)
    return np.array([lens[a] * lens[b] for a in range(k) for b in range(a + 1, k)], dtype=np.float64)


def test_split_is_equal_work_and_covers_every_pair():
    import numpy as np
    from paper_1512_07437_b300 import dist as qd
    import synth
    for fam in (synth.make_family("c2", 3), synth.make_family("c3", 1)):
        w = _work(fam.lengths.astype(np.int64))
        cum = np.concatenate([[0.0], np.cumsum(w)])
        for n in (1, 2, 3, 7, 8):
            b = qd.split_bounds(fam.offsets, n)
            assert b[0] == 0 and b[-1] == len(w) and (np.diff(b) > 0).all()
            parts = np.diff(cum[b])
            # every boundary is the one nearest to its share: a part is off the
            # ideal by at most one pair's work on either side
            assert np.abs(parts - cum[-1] / n).max() <= 2 * w.max()


def test_split_edge_cases():
    import numpy as np
    import pytest
    from paper_1512_07437_b300 import dist as qd
    from paper_1512_07437_b300.qp import QpError
    off = np.array([0, 3, 5, 9], dtype=np.int64)        # 3 sequences, 3 pairs
    assert qd.split_bounds(off, 3).tolist() == [0, 1, 2, 3]
    assert qd.split_bounds(off, 1).tolist() == [0, 3]
    with pytest.raises(QpError):
        qd.split_bounds(off, 4)                          # more parts than pairs
    with pytest.raises(QpError):
        qd.split_bounds(np.array([0, 3, 3], dtype=np.int64), 1)   # an empty sequence


def test_assemble_of_uneven_chunks_is_the_full_layout():
    """Single process: three ranges, one of them holding no entries at all."""
    import numpy as np
    from paper_1512_07437_b300 import dist as qd
    lens = [4, 1, 3, 2]
    full = _synthetic_result(lens, seed=9)
    # make pair 0 (4 x 1) hold no entry
    pro, pno = full["pair_row_off"], full["pair_nnz_off"]
    n0 = int(pno[1])
    full["row_ptr"][pro[0]:pro[1]] = 0
    full["col"], full["val"] = full["col"][n0:], full["val"][n0:]
    full["pair_nnz_off"] = np.concatenate([[0], pno[1:] - n0]).astype(np.int64)
    chunks = [_chunk_of(full, lens, a, b) for a, b in ((0, 1), (1, 4), (4, 6))]
    _same_layout(qd.assemble(chunks), full)
