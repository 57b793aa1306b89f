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
