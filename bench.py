"""Benchmark of the all-pairs posterior stage (one JSON line on stdout).

Workload (default, C3): one family of 500 synthetic protein sequences, lengths
150-500 (seeded evolution down a random binary tree, branch substitution
5-25%), all 124,750 pairs in one length-ordered persistent launch, FP32
scaled recurrences, threshold 0.01 CSR output and the MEA distance matrix.  A
step is one complete pass of the posterior stage over the family.

Metric: posterior-stage GCUPS = sum over pairs of m*n / step time / 1e9, where
one cell update is the whole per-cell work of pair-HMM forward and backward,
partition-function forward and backward, combination, threshold and MEA; and
the p50/p99 family latency of the serving loop.

  value : residues resident on the device, results left on the device;
          device time of each step (CUDA events on the launch stream), L2
          flushed (256 MiB write) before every step, outside the timed window.
  e2e   : host to host through the public API: residues from pinned host
          memory, qp_posteriors with host output (CSR, distances, MEA scores,
          log totals and flags all copied back to host memory; the library
          overlaps the copies of a large family with its computation by
          running it in pair ranges); wall time.
  e2e_csr_on_device : the same with the CSR left on the device and only the
          distance matrix read back (the guide tree's input).
  latency_ms / serving : the serving loop (qp_server_*: memory-admitted,
          device-resident, pairs of all admitted families batched into shared
          persistent launches) on the C4 trace: 200 families (10-1000
          sequences, log-uniform; lengths 50-1000) arriving as a Poisson
          process, run twice: at the configured 20 families/s, which offers
          more than the GPU serves (the capacity point), and with the same
          arrivals stretched to offer 70% of that capacity (the load point,
          whose latencies describe the loop rather than a backlog).
  c2, c5 : the same stage on the C2 family (64 sequences, 200-400) and the C5
          family (100 sequences, 2000-4000: long sequences, checkpointed form).
  f64_plain : the plain FP64 GPU form on the C1 and C2 families.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--config c1|c2|c3|c4|c5] [--precision f32|f64] [--no-legs] [--no-serving]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

ALU_OPS_PER_CELL = 61          # algorithmic FP32/INT issue slots per cell update
FLOPS_PER_CELL = 105           # the same work counted in flops (an FMA is 2)
BYTES_PER_CELL = 16            # stored design: (B_M, Zm_b) written in pass 1 and read in pass 2
FP64_NOMINAL_TFLOPS = 1.25     # B300 dense FP64, nominal (no measured FP64 peak is recorded)
FP32_LANES_PER_SM = 128
CONFIG_DESC = {
    "c1": "8 seqs, lengths 100-150, star tree s=0.30, 28 pairs",
    "c2": "64 seqs, lengths 200-400, star tree s=0.40, 2016 pairs",
    "c3": "500 seqs, lengths 150-500, random tree s~U[0.05,0.25], 124750 pairs",
    "c4": "serving: 200 families Poisson 20/s, 10-1000 seqs log-uniform, lengths 50-1000",
    "c5": "100 seqs, lengths 2000-4000, 3-domain roots, 4950 pairs",
}
# the sources of k_posterior_f32: a DRAM-traffic figure in profiles/ holds
# only while they are unchanged
# the translation units of k_posterior_f32 (its traffic record is keyed to them)
KERNEL_SOURCES = ["paper_1512_07437_b300/csrc/qp_f32.cuh", "paper_1512_07437_b300/csrc/qp_f32_w1.cu",
                  "paper_1512_07437_b300/csrc/qp_f32_w2.cu", "paper_1512_07437_b300/csrc/qp_internal.h"]
LOAD_FRACTION = 0.70           # offered load of the serving load point, of measured capacity
METRIC = "posterior-stage GCUPS and p50/p99 family latency, FP32 batched vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIG_DESC))
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="headline only (no c2/c5/serving/stage legs)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--subset", default="", metavar="K:MAXLEN",
                    help="profiling: only the first K sequences of length <= MAXLEN of the family")
    ap.add_argument("--variant", type=int, default=-1, help="profiling: force the kernel's register variant")
    ap.add_argument("--wpp", type=int, default=0, help="profiling: force the warps per pair (1 or 2)")
    ap.add_argument("--ckpt", type=int, default=-1,
                    help="profiling: force the stored (0) or the checkpointed (1) form of the FP32 kernel")
    ap.add_argument("--families", type=int, default=0,
                    help="profiling: serving trace of this many families (default: the C4 trace's 200)")
    ap.add_argument("--wpb", type=int, default=0,
                    help="profiling: force the block layout (2: one emission table, 8: 16 bank-sliced copies)")
    return ap.parse_args()


def subset_family(fam, spec: str):
    """The first K sequences of length <= MAXLEN of a family (spec "K:MAXLEN"),
    a reduced workload of the same family for profiler captures."""
    k, maxlen = (int(v) for v in spec.split(":"))
    keep = [a for a in range(fam.k) if fam.lengths[a] <= maxlen][:k]
    return synth.family_from_strings([fam.seq(a) for a in keep], name=f"{fam.name}-subset")


def dist_env():
    from paper_1512_07437_b300 import dist as qd
    return qd.env()


def kernel_src_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        p = os.path.join(ROOT, f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[0]) for s in self.samples if num(s[0]) is not None]
        mx = [num(s[1]) for s in self.samples if num(s[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for nm, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def recorded_traffic(key: str):
    """DRAM bytes of one k_posterior_f32 launch on workload ``key`` from the
    ncu summary in profiles/, or None when the kernel's sources changed since
    the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_posterior_f32_traffic.json")) as f:
            rec = json.load(f).get(key)
    except Exception:
        return None
    if not isinstance(rec, dict) or rec.get("kernel_src_sha") != kernel_src_sha():
        return None
    return rec.get("bytes")


def posterior_roofline(cells, kernel_ms, sm_count, max_mhz, traffic=None):
    """Roofline of k_posterior_f32: the lower of its two ceilings binds.
    HBM: the stored design (and the checkpointed one) moves 16 B per cell,
    (B_M, Zm_b) as two floats written in pass 1 and read back in pass 2, so
    the ceiling is the measured copy bandwidth / 16 B.  ALU: 61 issue slots
    per cell on 128 FP32 lanes per SM, so the ceiling is SMs x 128 x clock /
    61.  At 2032 MHz and 6.5 TB/s that is 631 against 407 Gcells/s: HBM."""
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    hbm_basis = "measured copy bandwidth (hbm_gbs), of measured"
    if not hbm:
        hbm, hbm_basis = 6400.0, "fallback 6.4 TB/s (no measured peak), of fallback"
    sec = kernel_ms * 1e-3
    alu_peak = sm_count * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12
    alu = {"achieved": cells * ALU_OPS_PER_CELL / sec / 1e12, "peak": alu_peak, "unit": "Tissue/s",
           "ops_per_cell": ALU_OPS_PER_CELL,
           "peak_basis": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz:.0f} MHz"}
    alu["frac"] = alu["achieved"] / alu_peak
    mem = {"achieved": cells * BYTES_PER_CELL / sec / 1e9, "peak": hbm, "unit": "GB/s",
           "bytes_per_cell": BYTES_PER_CELL, "peak_basis": hbm_basis}
    mem["frac"] = mem["achieved"] / hbm
    ceil = {"hbm": hbm * 1e9 / BYTES_PER_CELL / 1e9, "alu": alu_peak * 1e12 / ALU_OPS_PER_CELL / 1e9}
    top, other = (("hbm", mem), ("alu", alu)) if ceil["hbm"] <= ceil["alu"] else (("alu", alu), ("hbm", mem))
    out = {"bound": top[0], **top[1], "traffic": traffic, "ceilings_gcells_s": ceil, other[0]: other[1]}
    return out


def config_of(args, fam, prm) -> dict:
    """The workload as both arms report it."""
    return {"workload": f"{args.config}: {CONFIG_DESC[args.config]}", "seed": args.seed,
            "pairs": fam.n_pairs, "cells_per_step": fam.cells(), "threshold": prm.threshold,
            "combine": "rms", "precision": args.precision,
            "l2": "flushed (256 MiB write) before each timed step; per-step data far above L2"}


def cpu_baseline(fam, prm, budget_s: float, seed: int = 0):
    """The FP64 oracle on the host cores, on a bounded seeded sample of pairs:
    batches of seeded random pairs until about ``budget_s`` seconds of work;
    the rate is cells of the sample / its time."""
    import oracle
    pl = list(fam.pairs())
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(len(pl))
    threads = os.cpu_count() or 1
    L = fam.lengths.astype(np.int64)
    oracle.pairs(fam, [pl[order[-1]]], prm, threads=1)      # load the library
    batch = 4 * threads
    done, cells, dt = 0, 0.0, 0.0
    while dt < budget_s and done < len(order):
        sample = [pl[i] for i in order[done:done + batch]]
        t0 = time.perf_counter()
        oracle.pairs(fam, sample, prm, threads=threads)
        dt += time.perf_counter() - t0
        cells += float(sum(L[a] * L[b] for a, b in sample))
        done += len(sample)
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "sample": f"{done} seeded random pairs of the family ({cells:.3g} cells of {fam.cells():.3g}), "
                      f"FP64 log-space, {threads} threads, {dt:.1f} s; rate extrapolates by cells"}


def cpu_consistency(fam, prm, merges, seed: int, n_pairs: int = 12, T: int = 200, h: float = 3.0,
                    mem_bytes: float = 2.0 * 2**30):
    """The oracle's relaxation (dense FP64 products, numpy) on a few seeded
    pairs of the family that have selected third sequences, over the seeded
    guide tree ``merges``; its inputs are the oracle's own posteriors at the
    threshold, computed beforehand on a thread pool and not timed, and held
    in host memory: pairs whose inputs would take more than ``mem_bytes`` are
    not sampled.  The family's time is extrapolated by the dense work, sum
    over pairs and selected z of m l n."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    k = fam.k
    L = fam.lengths.astype(np.float64)
    d = oracle.tree_distances(merges, k)
    # dense work of every pair: m n sum_{z in Z} l_z
    work = np.zeros((k, k))
    for x in range(k):
        sel = (np.maximum(d[x][None, :], d) <= T)          # [y, z]: max(d_xz, d_zy) <= T
        sel[:, x] = False
        np.fill_diagonal(sel, False)
        work[x] = L[x] * L * (sel @ L)
    rng = np.random.Generator(np.random.PCG64(seed + 11))
    cand = [(x, y) for x, y in fam.pairs() if work[x, y] > 0]
    if not cand:
        return {"kind": "oracle", "sample": "no pair has a selected third sequence"}
    # the dense FP64 inputs are held in host memory: at most mem_bytes of them
    sample, need = [], set()
    for i in rng.permutation(len(cand)):
        if len(sample) == n_pairs:
            break
        x, y = cand[i]
        more = {(x, y)}
        for z in range(k):
            if z != x and z != y and max(d[x, z], d[z, y]) <= T:
                more.add((min(x, z), max(x, z)))
                more.add((min(z, y), max(z, y)))
        grown = need | more
        if 8.0 * sum(L[a] * L[b] for a, b in grown) > mem_bytes:
            continue
        sample.append((x, y))
        need = grown
    if not sample:
        return {"kind": "oracle", "sample": f"skipped: the oracle's dense inputs for one pair exceed "
                                            f"{mem_bytes / 2**30:.0f} GiB of host memory"}
    need = sorted(need)

    def dense(ab):
        P = oracle.pair(fam.codes(ab[0]), fam.codes(ab[1]), prm)["P"]
        return np.where(P >= prm.threshold, P, 0.0)
    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        S = dict(zip(need, ex.map(dense, need)))
    t0 = time.perf_counter()
    _, nz = oracle.consistency(S, [int(v) for v in fam.lengths], merges, T=T, h=h, theta=prm.threshold,
                               pairs=sample)
    dt = time.perf_counter() - t0
    w_sample = float(sum(work[x, y] for x, y in sample))
    w_all = float(sum(work[x, y] for x, y in fam.pairs()))
    return {"s_sample": dt, "family_s": dt * w_all / w_sample, "kind": "oracle", "cores": os.cpu_count() or 1,
            "sample": f"{len(sample)} seeded pairs with selected z ({sum(nz.values())} relaxations), dense "
                      f"FP64 products (numpy), seeded random guide tree, T={T}, h={h}; family time "
                      f"extrapolated by dense work (sum of m l n)"}


def run_reference(args, fam, prm, rank, config):
    """--impl reference: the FP64 oracle as it stands, on the host cores, each
    step a bounded seeded sample of the workload's pairs (about 3 s of host
    work); the rate extrapolates by cells."""
    if rank != 0:
        return
    import oracle
    threads = os.cpu_count() or 1
    pl = list(fam.pairs())
    rng = np.random.Generator(np.random.PCG64(args.seed + 100))
    L = fam.lengths.astype(np.int64)
    oracle.pairs(fam, [pl[0]], prm, threads=1)
    probe = [pl[i] for i in rng.permutation(len(pl))[:threads]]
    t0 = time.perf_counter()
    oracle.pairs(fam, probe, prm, threads=threads)
    rate = sum(L[a] * L[b] for a, b in probe) / max(time.perf_counter() - t0, 1e-3)
    step_cells = rate * 3.0          # about 3 s of host work per step
    times, cells_done = [], []
    for step in range(args.warmup + args.steps):
        sample, c = [], 0.0
        for i in rng.permutation(len(pl)):
            if c >= step_cells:
                break
            sample.append(pl[i])
            c += float(L[pl[i][0]] * L[pl[i][1]])
        t0 = time.perf_counter()
        oracle.pairs(fam, sample, prm, threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            cells_done.append(c)
    value = sum(cells_done) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                         "sample": f"seeded random pairs of the family, ~{statistics.mean(cells_done):.3g} "
                                   f"cells (about 3 s of host work) per step, FP64 log-space; "
                                   f"rate extrapolates by cells"},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving
def serve_trace(qp, torch, trace, prm, local, time_scale: float, warm_families: int = 3) -> dict:
    """Runs the serving loop on ``trace`` with arrival times multiplied by
    ``time_scale``: families are submitted from host memory at their arrival
    times, a poller thread collects results (the CSR stays on the device, the
    distance matrix is read back to pinned host memory).  Latency is submit to
    completion per family."""
    from paper_1512_07437_b300 import dist as qd
    dev = torch.device("cuda", local)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(min(0.55 * free, 150e9))
    srv = qp.Server(prm, budget, device=local, out_on_device=True)
    # warm-up: a few small families (allocator pool, autotuner, module load)
    warm = [synth.star_family(900 + i, 24, (200, 400), 0.3) for i in range(warm_families)]
    for f in warm:
        srv.poll(srv.submit(f.residues, f.offsets), -1).free()
    st0 = srv.stats()
    lat, lat_k = [], []
    pending = {}
    lock = threading.Lock()
    submitted = threading.Event()
    errors = []
    state = {"cells": 0.0, "fallbacks": 0, "t_last": 0.0}

    def poller():
        try:
            while True:
                with lock:
                    items = list(pending.items())
                if not items and submitted.is_set():
                    return
                hit = False
                for t, fam in items:
                    r = srv.poll(t, 0)
                    if r is None:
                        continue
                    hit = True
                    h_dist = torch.empty((fam.k, fam.k), dtype=torch.float32).pin_memory()
                    h_dist.copy_(r.dist)          # the guide tree's input comes back to the host
                    lat.append(r.kernel_ms[3])
                    lat_k.append((fam.k, r.kernel_ms[3], r.kernel_ms[0]))
                    state["cells"] += fam.cells()
                    state["fallbacks"] += r.n_fallback
                    r.free()
                    with lock:
                        del pending[t]
                    state["t_last"] = time.perf_counter()
                if not hit:
                    time.sleep(0.0005)
        except Exception as e:      # surfaced after the join
            errors.append(e)

    th = threading.Thread(target=poller, daemon=True)
    h2d = 0
    t0 = time.perf_counter()
    th.start()
    for t_arr, fam in trace:
        d = t0 + t_arr * time_scale - time.perf_counter()
        if d > 0:
            time.sleep(d)
        t = srv.submit(fam.residues, fam.offsets)
        h2d += int(fam.residues.nbytes + fam.offsets.nbytes)
        with lock:
            pending[t] = fam
    submitted.set()
    th.join()
    if errors:
        srv.destroy()
        raise errors[0]
    wall = state["t_last"] - t0
    st = srv.stats()
    srv.destroy()
    cells_rank = state["cells"]
    cells = qd.sum_over_ranks(cells_rank)
    wall = qd.max_over_ranks(wall)
    kernel_ms = st["kernel_ms"] - st0["kernel_ms"]
    lat_s = sorted(lat)

    def q(p):
        return lat_s[min(len(lat_s) - 1, int(round(p * (len(lat_s) - 1))))]
    span = trace[-1][0] * time_scale
    by_k = {}
    for name, lo, hi in (("k<50", 0, 50), ("50<=k<200", 50, 200), ("k>=200", 200, 1 << 30)):
        xs = sorted(l for k, l, _ in lat_k if lo <= k < hi)
        ws = sorted(w for k, _, w in lat_k if lo <= k < hi)
        if xs:
            by_k[name] = {"n": len(xs), "p50": xs[len(xs) // 2], "max": xs[-1],
                          "queued_p50": ws[len(ws) // 2]}
    return {
        "value": cells / wall / 1e9, "unit": "GCUPS", "families": len(trace),
        "arrival_rate_hz": len(trace) / span if span > 0 else None,
        "offered_gcups": cells_rank / span / 1e9 if span > 0 else None,
        "busy_gcups": cells_rank / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else None,
        "wall_s": wall, "cells": cells, "kernel_ms": kernel_ms,
        "latency_ms": {"p50": q(0.50), "p99": q(0.99), "max": lat_s[-1], "min": lat_s[0]},
        "latency_ms_by_k": by_k,
        "launches_f32": st["launches_f32"] - st0["launches_f32"],
        "launches_f64": st["launches_f64"] - st0["launches_f64"],
        "max_resident": st["max_resident"], "max_families_per_launch": st["max_families_per_launch"],
        "fp64_fallback_pairs": state["fallbacks"], "mem_budget_bytes": budget,
        "h2d_bytes": h2d, "d2h_bytes": int(sum(f.k * f.k * 4 for _, f in trace)),
    }


def serving_points(qp, torch, prm, local, rank, sm_count, max_mhz, n_families: int = 0):
    """The C4 trace at its configured arrival rate (the capacity point) and
    stretched to offer LOAD_FRACTION of the capacity measured there."""
    trace = synth.make_serving_trace(seed=4 + 1000 * rank, n_families=n_families or None)
    cap = serve_trace(qp, torch, trace, prm, local, 1.0)
    capacity = cap["busy_gcups"] or cap["value"]
    scale = cap["offered_gcups"] / (LOAD_FRACTION * capacity) if capacity else 1.0
    load = serve_trace(qp, torch, trace, prm, local, scale)
    for pt in (cap, load):
        pt["roofline"] = {**posterior_roofline(pt["cells"], pt["kernel_ms"], sm_count, max_mhz),
                          "kernel": "k_posterior_f32", "kernel_ms": pt["kernel_ms"]}
    load["time_scale"] = scale
    load["what"] = (f"the capacity point's arrivals stretched by {scale:.3f} to offer "
                    f"{LOAD_FRACTION:.0%} of its busy throughput")
    cap["what"] = "the trace at its configured 20 families/s (offered load above capacity: a backlog)"
    return {"workload": f"c4: {CONFIG_DESC['c4']}", "capacity_point": cap, "load_point": load,
            "latency_definition": "submit to completion per family (wall clock)",
            "value_definition": "cells of all families / wall time from the first arrival to the last completion"}


def run_serving(args, rank, world, local):
    """--config c4: the serving loop under Poisson arrivals (one trace per rank)."""
    import torch
    import paper_1512_07437_b300 as qp
    from paper_1512_07437_b300 import dist as qd
    torch.cuda.set_device(local)
    qd.init()
    dev = torch.device("cuda", local)
    prm = synth.default_params(threshold=0.01)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    with ClockSampler(local) as clk:
        sv = serving_points(qp, torch, prm, local, rank, sm_count, 2032.0, args.families)
    clocks = clk.summary()
    cap, load = sv["capacity_point"], sv["load_point"]
    line = {
        "metric": "posterior-stage GCUPS and p50/p99 family latency (serving)",
        "value": cap["value"], "unit": "GCUPS", "n_gpus": world, "steps": 1, "warmup": 3,
        "ms_per_step": 1e3 * cap["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"c4: {CONFIG_DESC['c4']}", "families": cap["families"],
                   "threshold": prm.threshold,
                   "l2": "inputs far larger than L2 (4e12 cells over 200 families)"},
        "latency_ms": {**load["latency_ms"], "at": f"load point ({LOAD_FRACTION:.0%} of capacity)",
                       "offered_gcups": load["offered_gcups"]},
        "serving": sv,
        "e2e": {"value": cap["value"], "unit": "GCUPS", "h2d_bytes_per_step": cap["h2d_bytes"],
                "d2h_bytes_per_step": cap["d2h_bytes"],
                "what": "families submitted from host memory at their arrival times; distance "
                        "matrices read back; wall time first arrival -> last completion"},
        "gpu_launches": int(cap["launches_f32"] + cap["launches_f64"] + 3 * cap["families"]),
        "roofline": cap["roofline"],
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    qd.finalize()


# ------------------------------------------------------------------ family legs
def timed_steps(torch, step, stream, flush, n):
    """Device time of n steps (CUDA events on the launch stream), L2 flushed
    before each, outside the timed window; returns (ms list, last results info)."""
    times, kms, fallbacks, nnz = [], [], 0, 0
    for _ in range(n):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kms.append(r.kernel_ms)
        fallbacks += r.n_fallback
        nnz = int(r.nnz)
        r.free()
    return times, kms, fallbacks, nnz


def event_kernel_ms(qp, step, local, flush, ki, n):
    """Device time of the posterior kernel alone: CUDA events around it on its
    stream, in a pass with plain launches (a captured graph carries none)."""
    qp.qp_set_option("graph", 0, device=local)
    try:
        out = []
        for _ in range(n):
            flush.zero_()
            r = step()
            out.append(r.kernel_ms[ki])
            r.free()
    finally:
        qp.qp_set_option("graph", 1, device=local)
    return out


def launch_config(qp, local):
    """The FP32 kernel's launch configuration the autotuner settled on."""
    return {k: qp.qp_get_counter(f"f32_{k}", device=local)
            for k in ("variant", "wpp", "warps_per_block", "tab_copies")}


def family_leg(qp, torch, fam, prm, local, stream, flush, steps, warmup, sm_count, max_mhz, key):
    """The stage on one family, device-resident, with its roofline."""
    dev = torch.device("cuda", local)
    params = qp.make_params(prm, device=local, stream=stream)
    d_res = torch.from_numpy(fam.residues).to(dev)

    def step():
        return qp.qp_posteriors(d_res, fam.offsets, params, out_on_device=True)
    # (the autotuner samples up to four launch configurations twice each on
    # the first calls of a launch shape)
    for _ in range(max(9, warmup)):
        step().free()
    torch.cuda.synchronize()
    ki = 0 if prm.precision == "f32" else 1
    times, kms, fallbacks, nnz = timed_steps(torch, step, stream, flush, steps)
    ev = event_kernel_ms(qp, step, local, flush, ki, max(3, min(steps, 5)))
    kernel_ms = statistics.mean(ev)
    ms = statistics.mean(times)
    out = {"workload": f"{key}: {CONFIG_DESC[key]}", "value": fam.cells() / (ms * 1e-3) / 1e9, "unit": "GCUPS",
           "ms_per_step": ms, "steps": steps, "pairs": fam.n_pairs, "cells_per_step": fam.cells(), "nnz": nnz,
           "fp64_fallback_pairs": fallbacks, "kernel_ms": kernel_ms,
           "kernel_ms_timed_region": statistics.mean(k[ki] for k in kms)}
    if prm.precision == "f32":
        out["roofline"] = {**posterior_roofline(fam.cells(), kernel_ms, sm_count, max_mhz,
                                                recorded_traffic(f"{key}-f32")),
                           "kernel": "k_posterior_f32", "kernel_ms": kernel_ms,
                           "launch": launch_config(qp, local)}
    del d_res
    return out


def f64_plain(qp, torch, fam, prm, local, stream, steps=3):
    """Device time of the plain FP64 GPU form on a family."""
    p64 = qp.make_params(prm.replace(precision="f64"), device=local, stream=stream)
    d_res = torch.from_numpy(fam.residues).to(torch.device("cuda", local))
    qp.qp_posteriors(d_res, fam.offsets, p64, out_on_device=True).free()
    ts, ks = [], []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = qp.qp_posteriors(d_res, fam.offsets, p64, out_on_device=True)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
        ks.append(r.kernel_ms[1])
        r.free()
    ms = statistics.mean(ts)
    ach = fam.cells() * FLOPS_PER_CELL / (ms * 1e-3) / 1e12
    return {"value": fam.cells() / (ms * 1e-3) / 1e9, "unit": "GCUPS", "ms_per_step": ms,
            "kernel_ms_timed_region": statistics.mean(ks), "steps": steps, "kernel": "k_posterior_f64",
            "pairs": fam.n_pairs, "cells_per_step": fam.cells(),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                         "frac": ach / FP64_NOMINAL_TFLOPS, "flops_per_cell": FLOPS_PER_CELL,
                         "peak_basis": "nominal B300 dense FP64 (not measured); step time"}}


def result_bytes(r) -> int:
    """Bytes of a result copied to host memory: CSR, distances, per-pair arrays."""
    P, k = int(r.n_pairs), int(r.k)
    b = 8 * (P + 1) * 2 + 4 * int(r.n_rows) + 8 * int(r.nnz) + 12 * k * k + 3 * 8 * P + 4 * P
    if r.precision == 1:
        b += 8 * int(r.nnz)
    return b


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.config == "c4":
        if args.impl == "reference":
            # the oracle on pairs of the trace's first families (same generator
            # seeds as the full trace), the family of median size
            fams = sorted((f for _, f in synth.make_serving_trace(seed=4, n_families=12)),
                          key=lambda f: f.cells())
            fam = fams[len(fams) // 2]
            prm = synth.default_params(threshold=0.01)
            return run_reference(args, fam, prm, rank, config_of(args, fam, prm))
        return run_serving(args, rank, world, local)
    from paper_1512_07437_b300 import dist as qd
    # every rank works on its own family of the configuration (weak scaling)
    fam = synth.make_family(args.config, qd.rank_seed(args.seed, rank))
    if args.subset:
        fam = subset_family(fam, args.subset)
    prm = synth.default_params(threshold=0.01, precision=args.precision)
    config = config_of(args, fam, prm)
    if args.subset:
        config["workload"] += f"; profiling subset {args.subset} ({fam.k} sequences)"
        config["pairs"], config["cells_per_step"] = fam.n_pairs, fam.cells()
    if args.impl == "reference":
        return run_reference(args, fam, prm, rank, config)

    import torch
    import paper_1512_07437_b300 as qp
    torch.cuda.set_device(local)
    qd.init()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cells = fam.cells()
    d_res = torch.from_numpy(fam.residues).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    params = qp.make_params(prm, device=local, stream=stream)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    if args.variant >= 0:
        qp.qp_set_option("variant", args.variant, device=local)
    if args.wpp > 0:
        qp.qp_set_option("wpp", args.wpp, device=local)
    if args.ckpt >= 0:
        qp.qp_set_option("ckpt", args.ckpt, device=local)
    if args.wpb > 0:
        qp.qp_set_option("warps_per_block", args.wpb, device=local)
        qp.qp_set_option("tab_copies", 16 if args.wpb >= 8 else 1, device=local)

    def step_dev():
        return qp.qp_posteriors(d_res, fam.offsets, params, out_on_device=True)

    ki = 0 if args.precision == "f32" else 1     # kernel_ms index of the posterior kernel
    # (the autotuner samples up to four launch configurations twice each on
    # the first calls of a launch shape: the warm-up covers them)
    warmup = max(9, args.warmup)
    for _ in range(warmup):
        step_dev().free()
    torch.cuda.synchronize()

    # ---- device-resident timing (the headline)
    cnt0 = {k: qp.qp_get_counter(k, device=local) for k in ("graph_captures", "graph_relaunches", "plain_calls")}
    qd.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times, kms, fallbacks, nnz = timed_steps(torch, step_dev, stream, flush, args.steps)
    torch.cuda.synchronize()
    qd.barrier()
    clocks = clk.summary()
    max_mhz = float(clocks["sm_max_mhz"] or peaks.get("sm_max_mhz", 2032.0))
    # one CUDA graph a step: k_encode, k_seqlogq, k_posterior_f32, k_posterior_f64
    # (follow-up, ends at once without fallbacks), k_scan_nnz, k_compact
    launches = 6 * args.steps
    graph_calls = {k: qp.qp_get_counter(k, device=local) - v for k, v in cnt0.items()}
    ms = statistics.mean(times)
    # whole job: cells of all ranks over the slowest rank's timed region
    value = qd.whole_job_rate(cells * args.steps, sum(times) / 1e3) / 1e9
    ev_kms = event_kernel_ms(qp, step_dev, local, flush, ki, max(3, min(args.steps, 8)))
    kernel_ms = statistics.mean(ev_kms)

    # ---- end to end, host to host through the public API: residues from
    # pinned host memory; qp_posteriors with host output copies every result
    # array (CSR, distances, MEA scores, log totals, flags) to host memory
    h_res = torch.from_numpy(fam.residues).pin_memory()
    n_e2e = max(3, min(args.steps // 2, 10))

    def e2e_host_step():
        r = qp.qp_posteriors(h_res.numpy(), fam.offsets, params, out_on_device=False)
        b = result_bytes(r)
        r.free()
        return b
    for _ in range(3):          # this call sequence captures and tunes on its first calls
        e2e_host_step()
    e2e_t, d2h = [], 0
    for _ in range(n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = e2e_host_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = qd.whole_job_rate(cells * len(e2e_t), sum(e2e_t)) / 1e9
    h2d = int(fam.residues.nbytes + fam.offsets.nbytes)

    # ---- end to end with the CSR left on the device (the next stages consume
    # it there) and the distance matrix read back to pinned host memory
    h_dist = torch.empty((fam.k, fam.k), dtype=torch.float32).pin_memory()

    def e2e_dev_step():
        r = qp.qp_posteriors(h_res.numpy(), fam.offsets, params, out_on_device=True)
        h_dist.copy_(r.dist, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        r.free()
    for _ in range(3):
        e2e_dev_step()
    e2d_t = []
    for _ in range(n_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_dev_step()
        e2d_t.append(time.perf_counter() - t0)
    e2d_val = qd.whole_job_rate(cells * len(e2d_t), sum(e2d_t)) / 1e9

    line = {
        "metric": METRIC,
        "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "f32" else "f64", "data": "synthetic",
        "config": config,
        "nnz": nnz, "fp64_fallback_pairs": fallbacks,
        "e2e": {"value": e2e_val, "unit": "GCUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * statistics.mean(e2e_t),
                "what": "host residues -> device; qp_posteriors host output: CSR, distances, MEA, "
                        "log totals and flags copied back to (pinned) host memory; wall time"},
        "e2e_csr_on_device": {"value": e2d_val, "unit": "GCUPS", "h2d_bytes_per_step": h2d,
                              "d2h_bytes_per_step": int(h_dist.numel() * 4),
                              "ms_per_step": 1e3 * statistics.mean(e2d_t),
                              "what": "host residues -> device; CSR kept on the device; distance matrix -> host"},
        "gpu_launches": launches,
        "graph_calls_in_timed_region": graph_calls,
        "clocks": clocks,
    }
    traffic = None if args.subset else recorded_traffic(f"{args.config}-{args.precision}")
    if args.precision == "f32":
        line["roofline"] = {**posterior_roofline(cells, kernel_ms, sm_count, max_mhz, traffic),
                            "kernel": "k_posterior_f32", "kernel_ms": kernel_ms,
                            "launch": launch_config(qp, local),
                            "kernel_ms_timed_region": statistics.mean(k[ki] for k in kms),
                            "kernel_timing": "CUDA events around the kernel (plain launches); "
                                             "kernel_ms_timed_region: the kernel's own time stamps in "
                                             "the graph steps",
                            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                              "(profiles/k_posterior_f32_traffic.json), null when the kernel "
                                              "changed since"}
    else:
        ach = cells * FLOPS_PER_CELL / (kernel_ms * 1e-3) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                            "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": traffic,
                            "peak_basis": "nominal B300 dense FP64 (not measured)",
                            "flops_per_cell": FLOPS_PER_CELL, "kernel": "k_posterior_f64",
                            "kernel_ms": kernel_ms}

    if not args.no_legs:
        legs(args, line, qp, torch, fam, prm, params, d_res, nnz, local, stream, flush, sm_count, max_mhz,
             rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(fam, prm, args.cpu_sample_s)
    if rank == 0:
        print(json.dumps(line), flush=True)
    qd.finalize()


def legs(args, line, qp, torch, fam, prm, params, d_res, nnz, local, stream, flush, sm_count, max_mhz,
         rank, world):
    """The other configurations and the stage's consumers, beside the headline."""
    from paper_1512_07437_b300 import dist as qd
    steps = max(3, min(args.steps, 10))
    seed = qd.rank_seed(args.seed, rank)
    for key in ("c2", "c5"):
        if key != args.config and args.precision == "f32":
            line[key] = family_leg(qp, torch, synth.make_family(key, seed), prm, local, stream, flush,
                                   steps, 3, sm_count, max_mhz, key)
    # FP32 batched vs plain FP64, on the families the FP64 form finishes quickly
    if args.precision == "f32":
        line["f64_plain"] = {key: f64_plain(qp, torch, synth.make_family(key, seed), prm, local, stream)
                             for key in ("c1", "c2")}
        line["f64_plain"]["c1"]["f32_same_family"] = family_leg(
            qp, torch, synth.make_family("c1", seed), prm, local, stream, flush, steps, 3, sm_count, max_mhz,
            "c1")["value"]

    # ---- entry budget: the same call with room for half of its entries (the
    # threshold is raised until they fit); extra passes over the entries at
    # the threshold T: the select reads the values twice (FP32 keys, 4 B; the
    # bits all keys share are known from the compaction), the filter reads the
    # values, then columns + values, and writes the kept N entries: about
    # 20 B x T + 8 B x N
    bpe = 8 if args.precision == "f32" else 16
    budget_bytes = max(bpe, (int(nnz) * bpe) // 2)
    params_b = qp.make_params(prm, device=local, stream=stream, entry_budget=budget_bytes)

    def step_b():
        return qp.qp_posteriors(d_res, fam.offsets, params_b, out_on_device=True)

    def step_plain():
        return qp.qp_posteriors(d_res, fam.offsets, params, out_on_device=True)
    for _ in range(3):
        step_b().free()
    b_times, _, _, b_nnz = timed_steps(torch, step_b, stream, flush, steps)
    rb = step_b()
    b_theta = rb.threshold_used
    rb.free()
    u_times, _, _, _ = timed_steps(torch, step_plain, stream, flush, steps)
    b_ms, u_ms = statistics.median(b_times), statistics.median(u_times)
    extra_ms = b_ms - u_ms
    extra_bytes = 20 * int(nnz) + 8 * b_nnz
    line["entry_budget"] = {
        "budget_bytes": budget_bytes, "threshold": prm.threshold, "threshold_used": b_theta,
        "nnz": b_nnz, "nnz_unbudgeted": int(nnz), "ms_per_step": b_ms, "ms_per_step_unbudgeted": u_ms,
        "extra_ms": extra_ms, "extra_bytes": extra_bytes,
        "extra_gbs": extra_bytes / (extra_ms * 1e-3) / 1e9 if extra_ms > 0 else None,
        "kernels": "k_sel_init, k_sel_hist (2 of 3 passes active), k_sel_pick, k_budget_count, "
                   "k_scan_nnz, k_budget_copy (plus the compaction into scratch)"}

    # ---- nucleotide mode: a family of the c2 shape over ACGT (64 sequences,
    # 200-400 nt, star tree, the same divergence) with GTR-derived tables
    nfam = synth.star_family(seed, 64, (200, 400), 0.40, keep=(200, 400), alphabet="nucleotide",
                             name="c2-nucleotide")
    nprm = synth.nucleotide_params(threshold=0.01, precision=args.precision)
    nuc = family_leg(qp, torch, nfam, nprm, local, stream, flush, steps, 3, sm_count, max_mhz, "c2")
    nuc["workload"] = "64 sequences over ACGT, 200-400 nt, star tree s=0.40, GTR-derived tables"
    line["nucleotide"] = nuc

    # ---- guide tree (weighted UPGMA) on the stage's FP64 distance matrix,
    # device to device, the step that consumes this stage's output
    r = step_plain()
    d64 = r.dist64.clone()
    r.free()
    tree_ms = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree = qp.qp_guide_tree(d64, stream=stream)
        e1.record(stream)
        e1.synchronize()
        tree_ms.append(e0.elapsed_time(e1))
    tree_host = (tree[0].cpu().numpy(), tree[1].cpu().numpy())
    line["guide_tree"] = {"k": fam.k, "ms": statistics.median(tree_ms[1:]),
                          "kernels": "k_tree_cluster (k up to about 660), else k_tree_mirror, "
                                     "k_tree_rows, k_tree_join",
                          "what": "weighted UPGMA on the FP64 distance matrix, device in and out"}

    # ---- selective consistency (stage III) on the stage's posteriors over
    # that guide tree, the paper's settings (T = 200, h = 3): device in and out
    post = step_plain()
    for _ in range(2):
        qp.qp_consistency(post, fam.offsets, tree[0], T=200, h=3.0, threshold=prm.threshold,
                          out_on_device=True).free()
    c_ms, c_dev_ms = [], []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc_ = qp.qp_consistency(post, fam.offsets, tree[0], T=200, h=3.0, threshold=prm.threshold,
                                out_on_device=True)
        e1.record(stream)
        e1.synchronize()
        c_ms.append(e0.elapsed_time(e1))
        c_dev_ms.append(rc_.kernel_ms[0])
        c_nnz = int(rc_.nnz)
        rc_.free()
    c_fma = qp.qp_get_counter("consistency_fma", device=local)
    c_form = qp.qp_get_counter("consistency_form", device=local)
    post.free()
    cms = statistics.median(c_ms)
    consistency = {"T": 200, "h": 3.0, "threshold": prm.threshold, "ms": cms,
                   "device_ms": statistics.median(c_dev_ms), "nnz_in": int(nnz), "nnz_out": c_nnz,
                   "fma": c_fma, "gflops": 2.0 * c_fma / (statistics.median(c_dev_ms) * 1e-3) / 1e9,
                   "form": "staged" if c_form == 1 else "row",
                   "kernels": "k_cons_tree, k_cons_ranges, k_cons_tcount/tscan/tfill, k_cons_interleave, "
                              + ("k_cons_stats, k_cons_relax_staged, " if c_form == 1 else "k_cons_relax, ")
                              + "k_cons_pair_nnz, k_scan_nnz, k_cons_compact"}
    peak_tops = sm_count * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12
    c_ach = 2.0 * consistency["fma"] / (consistency["device_ms"] * 1e-3) / 1e12
    consistency["roofline"] = {"bound": "alu", "achieved": c_ach, "peak": peak_tops, "unit": "Tissue/s",
                               "frac": c_ach / peak_tops, "ops_per_product": 2,
                               "kernel": "k_cons_relax_staged" if consistency["form"] == "staged" else "k_cons_relax",
                               "note": "scatter-bound: every product is a shared-memory atomic add"}
    line["consistency"] = consistency

    # ---- serving: the C4 trace at its capacity point and at 70% load
    if not args.no_serving and args.precision == "f32":
        sv = serving_points(qp, torch, prm, local, rank, sm_count, max_mhz)
        line["serving"] = sv
        load = sv["load_point"]
        line["latency_ms"] = {**load["latency_ms"], "at": f"serving load point ({LOAD_FRACTION:.0%} of capacity)",
                              "offered_gcups": load["offered_gcups"], "served_gcups": load["value"],
                              "capacity_point": {**sv["capacity_point"]["latency_ms"],
                                                 "offered_gcups": sv["capacity_point"]["offered_gcups"],
                                                 "served_gcups": sv["capacity_point"]["value"]}}
        line["gpu_launches_serving"] = int(sum(sv[p]["launches_f32"] + sv[p]["launches_f64"]
                                               for p in ("capacity_point", "load_point")))

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref_tree = oracle.guide_tree(d64.cpu().numpy())
        line["cpu_guide_tree"] = {
            "s": time.perf_counter() - t0, "kind": "oracle", "k": fam.k,
            "identical": bool(np.array_equal(ref_tree["merges"], tree_host[0])
                              and np.array_equal(ref_tree["heights"], tree_host[1]))}
        syn_tree = synth.random_guide_tree(args.seed + 7, fam.k)
        line["cpu_consistency"] = cpu_consistency(fam, prm, syn_tree, args.seed, n_pairs=4)


if __name__ == "__main__":
    main()
