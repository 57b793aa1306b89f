"""Oracle for the all-pairs posterior stage -- TEST INFRASTRUCTURE ONLY.

Plain FP64 log-space CPU implementation (``oracle.c``) of what the posterior
stage computes (paper, Methods, stage I): pair-HMM and partition-function
posteriors, their combination, the sparse matrix at threshold theta, the MEA
score and the MEA distance.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA path and imports nothing from
it; both sides take their inputs from ``synth`` only.

Every function here is pinned by tests against brute-force enumeration,
closed forms, limits and invariants (tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

COMBINE = {"rms": 0, "mean": 1, "hmm": 2, "pf": 3}
# residue letters -> codes: the 20 amino acids, or the nucleotide mode's
# A, C, G, T with U read as T (paper, Methods, "Other algorithmic
# improvements": nucleotide mode)
_LUTS = {}
for _name, _letters in (("protein", "ACDEFGHIKLMNPQRSTVWY"), ("nucleotide", "ACGT")):
    _t = np.full(256, 255, dtype=np.uint8)
    for _i, _c in enumerate(_letters):
        _t[ord(_c)] = _i
        _t[ord(_c.lower())] = _i
    _LUTS[_name] = _t
_LUTS["nucleotide"][[ord("U"), ord("u")]] = 3
_LUT = _LUTS["protein"]


class OrParams(ctypes.Structure):
    _fields_ = [
        ("pi", ctypes.c_double * 5),
        ("delta1", ctypes.c_double), ("eps1", ctypes.c_double),
        ("delta2", ctypes.c_double), ("eps2", ctypes.c_double),
        ("emit_pair", ctypes.c_double * 400),
        ("emit_bg", ctypes.c_double * 20),
        ("end_w", ctypes.c_double * 5),
        ("score", ctypes.c_double * 400),
        ("gap_open", ctypes.c_double), ("gap_ext", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("combine", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.or_pair.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int,
                                    ctypes.POINTER(OrParams), dp, dp, dp, dp, dp,
                                    dp, dp, dp, dp, dp]
            lib.or_pair.restype = ctypes.c_int
            lib.or_pairs.argtypes = [u8p, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                     ctypes.POINTER(OrParams), ctypes.c_double,
                                     ctypes.c_int, dp, dp, dp,
                                     ctypes.POINTER(ctypes.c_int64)]
            lib.or_pairs.restype = ctypes.c_int
            _lib = lib
    return _lib


def to_struct(prm) -> OrParams:
    """Copy a synth.ModelParams into the oracle's own parameter layout."""
    s = OrParams()
    s.pi[:] = [float(v) for v in prm.pi]
    s.delta1, s.eps1 = float(prm.delta1), float(prm.eps1)
    s.delta2, s.eps2 = float(prm.delta2), float(prm.eps2)
    s.emit_pair[:] = [float(v) for v in np.asarray(prm.emit_pair).reshape(-1)]
    s.emit_bg[:] = [float(v) for v in prm.emit_bg]
    s.end_w[:] = [float(v) for v in prm.end_w]
    s.score[:] = [float(v) for v in np.asarray(prm.score).reshape(-1)]
    s.gap_open, s.gap_ext = float(prm.gap_open), float(prm.gap_ext)
    s.temperature = float(prm.temperature)
    s.combine = COMBINE[prm.combine] if isinstance(prm.combine, str) else int(prm.combine)
    return s


def encode(seq, alphabet: str = "protein") -> np.ndarray:
    """Residue letters (str or uint8 ASCII array) -> codes: 0..19 for
    proteins, 0..3 (A, C, G, T; U as T) for nucleotides."""
    if isinstance(seq, str):
        seq = np.frombuffer(seq.encode("ascii"), dtype=np.uint8)
    c = _LUTS[alphabet][np.asarray(seq, dtype=np.uint8)]
    if (c == 255).any():
        raise ValueError(f"residue outside the {alphabet} alphabet")
    return c


def _as_codes(s) -> np.ndarray:
    """Letters (str / ASCII bytes) or an array of codes 0..19 -> codes."""
    if isinstance(s, np.ndarray) and s.dtype != np.uint8:
        s = s.astype(np.uint8)
    if isinstance(s, np.ndarray) and s.size and int(s.max()) < 20:
        return np.ascontiguousarray(s, dtype=np.uint8)
    return np.ascontiguousarray(encode(s), dtype=np.uint8)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def pair(x, y, prm) -> dict:
    """All outputs of one pair (x, y are residue codes or letters)."""
    lib = _load()
    x = _as_codes(x)
    y = _as_codes(y)
    m, n = int(x.size), int(y.size)
    if m < 1 or n < 1:
        raise ValueError("empty sequence")
    st = to_struct(prm)
    out = {k: np.zeros((m, n)) for k in ("P_hmm", "P_pf", "P")}
    gx_h, gy_h, gx_p, gy_p = np.zeros(m), np.zeros(n), np.zeros(m), np.zeros(n)
    logz = np.zeros(4)
    mea = np.zeros(1)
    dist = np.zeros(1)
    dp = ctypes.c_double
    rc = lib.or_pair(_ptr(x, ctypes.c_uint8), m, _ptr(y, ctypes.c_uint8), n,
                     ctypes.byref(st), _ptr(out["P_hmm"], dp), _ptr(out["P_pf"], dp),
                     _ptr(out["P"], dp), _ptr(gx_h, dp), _ptr(gy_h, dp),
                     _ptr(gx_p, dp), _ptr(gy_p, dp), _ptr(logz, dp),
                     _ptr(mea, dp), _ptr(dist, dp))
    if rc != 0:
        raise MemoryError("oracle: out of memory")
    out.update(gx_hmm=gx_h, gy_hmm=gy_h, gx_pf=gx_p, gy_pf=gy_p,
               logz_hmm=logz[0], logz_hmm_bwd=logz[1], logz_pf=logz[2],
               logz_pf_bwd=logz[3], mea=float(mea[0]), dist=float(dist[0]))
    return out


def sparsify(P: np.ndarray, theta: float):
    """Entries with P >= theta as CSR (row_ptr, col, val), columns ascending."""
    m = P.shape[0]
    keep = P >= theta
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(keep.sum(axis=1))
    rows, cols = np.nonzero(keep)
    return row_ptr, cols.astype(np.int64), P[rows, cols]


def budget_threshold(values, theta: float, n_keep: int, dtype=np.float32):
    """Threshold of the entry budget (paper, Methods, "Other algorithmic
    improvements": the posterior matrices are fitted into a user-given amount
    of memory by lowering the sparsity coefficient, i.e. keeping fewer
    entries).

    ``values``: every entry kept at threshold ``theta`` (all >= theta), taken
    in the precision the entries are compared in (``dtype``).  ``n_keep``: the
    entries the budget holds.  Returns the smallest threshold t >= theta in
    that precision with count(values >= t) <= n_keep: theta itself when the
    entries already fit, else the next representable value above the
    (n_keep + 1)-th largest value (all entries equal to it are dropped).
    """
    v = np.asarray(values, dtype=dtype).ravel()
    t0 = dtype(theta)
    if v.size <= n_keep:
        return t0
    largest_first = np.sort(v)[::-1]
    return np.nextafter(largest_first[n_keep], dtype(np.inf))


def tree_distances(merges, k: int) -> np.ndarray:
    """Tree-guided distance of selective consistency (paper, Methods,
    "Selective consistency", variant (b)): d[x, y] = the number of sequences
    (leaves) in the smallest subtree of the guide tree that contains both x
    and y, i.e. the subtree at their lowest common ancestor.  ``merges`` are
    the joins of the guide tree (leaves 0..k-1, the node of step s is k + s).
    d[x, x] = 1."""
    members = {i: [i] for i in range(k)}
    d = np.ones((k, k), dtype=np.int64)
    for s, (a, b) in enumerate(np.asarray(merges, dtype=np.int64).reshape(-1, 2)):
        A, B = members.pop(int(a)), members.pop(int(b))
        size = len(A) + len(B)
        for x in A:
            for y in B:
                d[x, y] = d[y, x] = size
        members[k + s] = A + B
    return d


def consistency(S: dict, lens, merges, T: int = 200, h: float = 3.0, n_max: int = 200,
                theta: float = 0.01, pairs=None) -> dict:
    """Selective consistency (paper, Methods, stage III and "Selective
    consistency"): every posterior matrix S_xy is relaxed through the third
    sequences z whose tree distances to x and y both stay within T, and its
    own signal is amplified by h_xy.

    ``S``: {(x, y): dense (len x, len y) matrix} for every pair x < y (the
    sparse posteriors, zeros where absent); S_yx is S_xy transposed.
    For each pair, with Z = {z not in {x, y} : max(d_xz, d_zy) <= T} and
    h_xy = 1 + (h - 1) min(|Z|, n_max) / n_max:
        S'_xy = (2 h_xy S_xy + sum_{z in Z} S_xz S_zy) / (2 + |Z|),
    the relaxation of ProbCons (a sum over all sequences, x and y included
    with S_xx = I, divided by their number) restricted to Z; then entries
    below ``theta`` are dropped.  Returns {(x, y): dense S'_xy} and
    {(x, y): |Z|}.  ``pairs``: relax only these (x, y), x < y (``S`` then
    needs only the matrices they use)."""
    k = len(lens)
    d = tree_distances(merges, k)

    def mat(a, b):
        return S[(a, b)] if a < b else S[(b, a)].T

    if pairs is None:
        pairs = [(x, y) for x in range(k) for y in range(x + 1, k)]
    out, nz = {}, {}
    for x, y in pairs:
        Z = [z for z in range(k) if z != x and z != y and max(d[x, z], d[z, y]) <= T]
        hxy = 1.0 + (h - 1.0) * min(len(Z), n_max) / n_max
        acc = 2.0 * hxy * S[(x, y)]
        for z in Z:
            acc = acc + mat(x, z) @ mat(z, y)
        R = acc / (2.0 + len(Z))
        R[R < theta] = 0.0
        out[(x, y)] = R
        nz[(x, y)] = len(Z)
    return out, nz


def pairs(family, pair_list, prm, threads: int | None = None, theta: float | None = None) -> dict:
    """Per-pair log Z (HMM, PF), MEA score, distance and nnz for the listed
    pairs of ``family``, on a thread pool of ``threads`` host cores."""
    lib = _load()
    threads = os.cpu_count() if threads is None else threads
    codes = encode(family.residues, getattr(family, "alphabet", "protein"))
    off = np.ascontiguousarray(family.offsets, dtype=np.int64)
    pl = np.asarray(list(pair_list), dtype=np.int32).reshape(-1, 2)
    pa = np.ascontiguousarray(pl[:, 0])
    pb = np.ascontiguousarray(pl[:, 1])
    npairs = pl.shape[0]
    logz = np.zeros(2 * npairs)
    mea = np.zeros(npairs)
    dist = np.zeros(npairs)
    nnz = np.zeros(npairs, dtype=np.int64)
    theta = prm.threshold if theta is None else theta
    st = to_struct(prm)
    dp = ctypes.c_double
    rc = lib.or_pairs(_ptr(codes, ctypes.c_uint8), _ptr(off, ctypes.c_int64),
                      _ptr(pa, ctypes.c_int32), _ptr(pb, ctypes.c_int32), npairs,
                      ctypes.byref(st), float(theta), int(threads), _ptr(logz, dp),
                      _ptr(mea, dp), _ptr(dist, dp), _ptr(nnz, ctypes.c_int64))
    if rc != 0:
        raise MemoryError("oracle: out of memory")
    return dict(logz_hmm=logz[0::2].copy(), logz_pf=logz[1::2].copy(), mea=mea,
                dist=dist, nnz=nnz, threads=threads)


def guide_tree(dist) -> dict:
    """Guide tree by weighted UPGMA (paper, Methods, stage II: the pairwise
    distances of stage I feed weighted UPGMA, after Sneath and Sokal).

    Weighted UPGMA (WPGMA): repeatedly join the two clusters at the smallest
    distance; the distance from the joined cluster to any other cluster is
    the mean of the distances from its two parts, whatever their sizes.
    Clusters live in slots 0..k-1 (slot i starts as leaf i); joining the
    clusters in slots i < j puts the new cluster in slot i and empties slot j.
    Ties: the smallest distance, then the smallest i, then the smallest j.
    Leaves have ids 0..k-1, the cluster formed at step s has id k + s.

    Returns merges (k-1, 2) int32 (ids joined at each step) and heights
    (k-1,) float64 (half the joining distance).  Plain O(k^3) (a full
    search of the live pairs at every step), FP64.
    """
    D = np.array(dist, dtype=np.float64)
    k = D.shape[0]
    if D.shape != (k, k) or k < 2:
        raise ValueError("dist must be a k x k matrix with k >= 2")
    alive = np.ones(k, dtype=bool)
    cid = np.arange(k)
    merges = np.zeros((k - 1, 2), dtype=np.int32)
    heights = np.zeros(k - 1)
    upper = np.triu(np.ones((k, k), dtype=bool), 1)
    for s in range(k - 1):
        # candidate pairs i < j among live slots; the first minimum in
        # row-major order is the tie rule (smallest i, then smallest j)
        cand = np.where(upper & alive[:, None] & alive[None, :], D, np.inf)
        bi, bj = divmod(int(np.argmin(cand)), k)
        best = cand[bi, bj]
        merges[s] = (cid[bi], cid[bj])
        heights[s] = best / 2.0
        others = alive.copy()
        others[bi] = others[bj] = False
        v = (D[bi, others] + D[bj, others]) / 2.0
        D[bi, others] = v
        D[others, bi] = v
        alive[bj] = False
        cid[bi] = k + s
    return dict(merges=merges, heights=heights)
