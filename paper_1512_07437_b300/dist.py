"""Multi-GPU host logic: one process per GPU.

The pairs of the posterior stage are independent (paper, Methods, stage I),
so ranks share nothing while they compute.  Two ways to use several GPUs:

  * independent families per rank (weak scaling): ranks meet only to agree
    on timing -- a barrier on both sides of the timed region, the maximum of
    the per-rank times, and sums of the work done;
  * one family split over the ranks: qp_split_pairs cuts the linear pair
    order into contiguous ranges of equal work (cumulative sum of m n), each
    rank computes its range (qp_posteriors_range), and one gather rebuilds the
    single-rank layout of the result bit for bit: per-pair CSR blocks and
    per-pair values are concatenated in range order with their offsets
    shifted, and the distance matrices, whose entries each come from exactly
    one rank, are summed.

The process group is NCCL with GPUs, gloo on CPU.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> bool:
    """Joins the process group when world_size > 1; returns whether it did."""
    import torch
    import torch.distributed as dist
    _, world, _ = env()
    if world <= 1 or dist.is_initialized():
        return dist.is_initialized()
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return True


def _reduce(x: float, op) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


def barrier():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


def rank_seed(base: int, rank: int) -> int:
    """Seed of the synthetic workload of a rank (distinct per rank)."""
    return int(base) + 7919 * int(rank)


def whole_job_rate(units_this_rank: float, seconds_this_rank: float) -> float:
    """Units of all ranks over the slowest rank's time (units per second)."""
    units = sum_over_ranks(units_this_rank)
    secs = max_over_ranks(seconds_this_rank)
    return units / secs if secs > 0 else 0.0


def finalize():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


# ---------------------------------------------------------------- one family over several ranks
# Per-pair arrays of a result, concatenated in range order by the gather.
PAIR_FIELDS = ("mea", "log_z_hmm", "log_z_pf", "pair_flags")


def split_bounds(offsets, world: int):
    """Pair ranges of equal work, one per rank (qp_split_pairs)."""
    from .qp import qp_split_pairs
    return qp_split_pairs(offsets, world)


def result_chunk(res) -> dict:
    """The arrays of a (range) result that the gather moves, as host numpy
    arrays: the CSR (pair_row_off, row_ptr, pair_nnz_off, col, val and val64
    when present), the per-pair values and the k x k distance matrices."""
    import numpy as np

    def h(x):
        return None if x is None else (x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)).copy()
    out = {name: h(res.array(name)) for name in ("pair_row_off", "row_ptr", "pair_nnz_off", "col", "val",
                                                 "val64", "dist", "dist64") + PAIR_FIELDS}
    if out["val64"] is None:
        del out["val64"]
    return out


def assemble(chunks) -> dict:
    """The family's single-rank layout from the chunks of consecutive pair
    ranges (in range order): row and entry offsets are shifted by the rows
    and entries of the chunks before, everything per pair or per row is
    concatenated, and the distance matrices are summed (each entry is set by
    exactly one chunk, so the sum is exact)."""
    import numpy as np
    pro, pno = [np.zeros(1, dtype=np.int64)], [np.zeros(1, dtype=np.int64)]
    rows = nnz = 0
    for c in chunks:
        pro.append(c["pair_row_off"][1:] + rows)
        pno.append(c["pair_nnz_off"][1:] + nnz)
        rows += int(c["pair_row_off"][-1])
        nnz += int(c["pair_nnz_off"][-1])
    out = {"pair_row_off": np.concatenate(pro), "pair_nnz_off": np.concatenate(pno)}
    for name in ("row_ptr", "col", "val", "val64") + PAIR_FIELDS:
        if name in chunks[0]:
            out[name] = np.concatenate([c[name] for c in chunks])
    for name in ("dist", "dist64"):
        acc = chunks[0][name].copy()
        for c in chunks[1:]:
            acc += c[name]
        out[name] = acc
    return out


def _gather_var(x, world: int, dev):
    """All-gather of a 1-D array whose length differs per rank (padded to the
    longest); returns the per-rank numpy arrays."""
    import numpy as np
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dev)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    ns = [int(v.item()) for v in ns]
    m = max(ns)
    if m == 0:
        return [np.zeros(0, dtype=np.asarray(x).dtype) for _ in range(world)]
    pad = torch.zeros(m, dtype=t.dtype, device=dev)
    pad[:t.numel()] = t
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return [parts[r][:ns[r]].cpu().numpy() for r in range(world)]


def gather_chunks(chunk: dict, dst: int = 0):
    """Collective: every rank passes the chunk of its pair range (ranks in
    range order); rank dst gets the assembled single-rank layout, the others
    None.  Without a process group the chunk is the whole result."""
    import numpy as np
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return assemble([chunk])
    world, rank = dist.get_world_size(), dist.get_rank()
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    parts = {name: _gather_var(arr, world, dev) for name, arr in chunk.items() if name not in ("dist", "dist64")}
    sums = {}
    for name in ("dist", "dist64"):
        t = torch.from_numpy(np.ascontiguousarray(chunk[name])).to(dev)
        dist.reduce(t, dst, op=dist.ReduceOp.SUM)
        sums[name] = t.cpu().numpy()
    if rank != dst:
        return None
    chunks = [{name: parts[name][r] for name in parts} for r in range(world)]
    for r in range(world):
        chunks[r]["dist"] = sums["dist"] if r == 0 else np.zeros_like(sums["dist"])
        chunks[r]["dist64"] = sums["dist64"] if r == 0 else np.zeros_like(sums["dist64"])
    return assemble(chunks)


def posteriors_split(residues, offsets, params, dst: int = 0, out_on_device: bool = True):
    """The posterior stage of one family over every rank of the process
    group: this rank's equal-work pair range on its GPU, then one gather;
    rank dst returns the family's result arrays (numpy, the single-rank
    layout), the other ranks None."""
    from .qp import qp_posteriors_range
    rank, world, _ = env()
    bounds = split_bounds(offsets, world)
    res = qp_posteriors_range(residues, offsets, params, int(bounds[rank]), int(bounds[rank + 1]),
                              out_on_device=out_on_device)
    chunk = result_chunk(res)
    res.free()
    return gather_chunks(chunk, dst)
