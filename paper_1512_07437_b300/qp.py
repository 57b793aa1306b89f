"""ctypes binding of libqp.so (include/qp.h), same names as the C entry points.

Argument marshalling only: every step of the posterior stage runs in the
library's CUDA kernels.  There is no fallback: if libqp.so is missing or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqp.so")

QP_OK, QP_EINVAL, QP_ENOMEM, QP_ECUDA, QP_ETIMEOUT, QP_ECANCELLED, QP_ENOTREADY = range(7)
QP_COMBINE = {"rms": 0, "mean": 1, "hmm": 2, "pf": 3}
QP_PRECISION = {"f32": 0, "f64": 1}
QP_ALPHABET = {"protein": 0, "nucleotide": 1}
QP_F32_SCALED, QP_F64_PLAIN = 0, 1
_STATUS_NAMES = {0: "QP_OK", 1: "QP_EINVAL", 2: "QP_ENOMEM", 3: "QP_ECUDA",
                 4: "QP_ETIMEOUT", 5: "QP_ECANCELLED", 6: "QP_ENOTREADY"}
GUARD_BITS = {2: "range", 3: "gap", 4: "factor", 5: "post", 6: "agree_hmm", 7: "agree_pf",
              8: "total", 9: "corner", 10: "stage", 11: "pool"}


class QpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class qp_family(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("residues_on_device", ctypes.c_int32),
                ("residues", ctypes.c_void_p), ("offsets", ctypes.POINTER(ctypes.c_int64))]


class qp_params(ctypes.Structure):
    _fields_ = [
        ("pi", ctypes.c_double * 5),
        ("delta1", ctypes.c_double), ("eps1", ctypes.c_double),
        ("delta2", ctypes.c_double), ("eps2", ctypes.c_double),
        ("emit_pair", ctypes.c_double * 400), ("emit_bg", ctypes.c_double * 20),
        ("end_w", ctypes.c_double * 5), ("score", ctypes.c_double * 400),
        ("gap_open", ctypes.c_double), ("gap_ext", ctypes.c_double),
        ("temperature", ctypes.c_double),
        ("end_gap_mode", ctypes.c_int32), ("combine", ctypes.c_int32),
        ("threshold", ctypes.c_double),
        ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
        ("stream", ctypes.c_void_p), ("entry_budget", ctypes.c_int64),
        ("alphabet", ctypes.c_int32), ("reserved_", ctypes.c_int32),
    ]


class qp_result(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32), ("on_device", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
        ("n_pairs", ctypes.c_int64), ("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("pair_row_off", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
        ("pair_nnz_off", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("val", ctypes.c_void_p), ("val64", ctypes.c_void_p),
        ("dist", ctypes.c_void_p), ("dist64", ctypes.c_void_p),
        ("mea", ctypes.c_void_p), ("log_z_hmm", ctypes.c_void_p),
        ("log_z_pf", ctypes.c_void_p), ("pair_flags", ctypes.c_void_p),
        ("kernel_ms", ctypes.c_double * 4), ("n_fallback", ctypes.c_int64),
        ("guard_info", ctypes.c_int32 * 12), ("threshold_used", ctypes.c_double),
        ("owner_", ctypes.c_void_p),
    ]


class qp_consistency_params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("n_max", ctypes.c_int32), ("h", ctypes.c_double),
                ("threshold", ctypes.c_double)]


class qp_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
        ("pairs_done", ctypes.c_int64), ("cells_done", ctypes.c_double),
        ("launches_f32", ctypes.c_int64), ("launches_f64", ctypes.c_int64),
        ("kernel_ms", ctypes.c_double),
        ("resident", ctypes.c_int32), ("max_resident", ctypes.c_int32),
        ("max_families_per_launch", ctypes.c_int32), ("queued", ctypes.c_int32),
        ("reserved_bytes", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
    ]


_lib = None


def lib():
    """Loads libqp.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1512_07437_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.qp_posteriors.argtypes = [P(qp_family), P(qp_params), ctypes.c_int32, P(P(qp_result))]
        L.qp_posteriors.restype = ctypes.c_int
        L.qp_posteriors_range.argtypes = [P(qp_family), P(qp_params), ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int32, P(P(qp_result))]
        L.qp_posteriors_range.restype = ctypes.c_int
        L.qp_split_pairs.argtypes = [ctypes.c_int32, P(ctypes.c_int64), ctypes.c_int32, P(ctypes.c_int64)]
        L.qp_split_pairs.restype = ctypes.c_int
        L.qp_result_free.argtypes = [P(qp_result)]
        L.qp_result_free.restype = None
        L.qp_last_error.restype = ctypes.c_char_p
        L.qp_version.restype = ctypes.c_char_p
        L.qp_server_create.argtypes = [P(qp_params), ctypes.c_size_t, ctypes.c_int32, P(ctypes.c_void_p)]
        L.qp_server_create.restype = ctypes.c_int
        L.qp_server_submit.argtypes = [ctypes.c_void_p, P(qp_family), P(ctypes.c_uint64)]
        L.qp_server_submit.restype = ctypes.c_int
        L.qp_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, P(P(qp_result))]
        L.qp_server_poll.restype = ctypes.c_int
        L.qp_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.qp_server_cancel.restype = ctypes.c_int
        L.qp_set_option.argtypes = [ctypes.c_int32, ctypes.c_char_p, ctypes.c_int64]
        L.qp_set_option.restype = ctypes.c_int
        L.qp_get_counter.argtypes = [ctypes.c_int32, ctypes.c_char_p, P(ctypes.c_int64)]
        L.qp_get_counter.restype = ctypes.c_int
        L.qp_server_get_stats.argtypes = [ctypes.c_void_p, P(qp_server_stats)]
        L.qp_server_get_stats.restype = ctypes.c_int
        L.qp_server_destroy.argtypes = [ctypes.c_void_p]
        L.qp_server_destroy.restype = None
        L.qp_pair_posteriors_static.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                P(qp_params), ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                P(ctypes.c_int64)]
        L.qp_pair_posteriors_static.restype = ctypes.c_int
        L.qp_guide_tree.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.qp_guide_tree.restype = ctypes.c_int
        L.qp_consistency.argtypes = [P(qp_result), P(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int32,
                                     P(qp_consistency_params), ctypes.c_int32, P(P(qp_result))]
        L.qp_consistency.restype = ctypes.c_int
        _lib = L
    return _lib


def qp_last_error() -> str:
    return lib().qp_last_error().decode()


def qp_version() -> str:
    return lib().qp_version().decode()


def _check(rc: int):
    if rc != QP_OK:
        raise QpError(rc, qp_last_error())


def make_params(prm, device: int = 0, stream=None, threshold: Optional[float] = None,
                combine: Optional[str] = None, precision: Optional[str] = None,
                entry_budget: Optional[int] = None) -> qp_params:
    """qp_params from any object with the model fields (pi, delta1, ...).
    ``entry_budget``: bytes the sparse entries may take (0: no budget)."""
    p = qp_params()
    p.pi[:] = [float(v) for v in prm.pi]
    p.delta1, p.eps1 = float(prm.delta1), float(prm.eps1)
    p.delta2, p.eps2 = float(prm.delta2), float(prm.eps2)
    p.emit_pair[:] = [float(v) for v in np.asarray(prm.emit_pair).reshape(-1)]
    p.emit_bg[:] = [float(v) for v in prm.emit_bg]
    p.end_w[:] = [float(v) for v in prm.end_w]
    p.score[:] = [float(v) for v in np.asarray(prm.score).reshape(-1)]
    p.gap_open, p.gap_ext = float(prm.gap_open), float(prm.gap_ext)
    p.temperature = float(prm.temperature)
    p.end_gap_mode = int(getattr(prm, "end_gap_mode", 0))
    c = combine if combine is not None else prm.combine
    p.combine = QP_COMBINE[c] if isinstance(c, str) else int(c)
    p.threshold = float(threshold if threshold is not None else prm.threshold)
    pr = precision if precision is not None else prm.precision
    p.precision = QP_PRECISION[pr] if isinstance(pr, str) else int(pr)
    p.device = int(device)
    p.entry_budget = int(entry_budget if entry_budget is not None else getattr(prm, "entry_budget", 0))
    al = getattr(prm, "alphabet", "protein")
    p.alphabet = QP_ALPHABET[al] if isinstance(al, str) else int(al)
    if stream is None:
        p.stream = None
    elif isinstance(stream, int):
        p.stream = stream
    else:   # torch.cuda.Stream
        p.stream = int(stream.cuda_stream)
    return p


def make_family(residues, offsets) -> tuple:
    """qp_family from residues (numpy uint8 host array, or a torch CUDA uint8
    tensor) and host int64 offsets.  Returns (struct, keep-alive tuple)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    f = qp_family()
    f.k = int(off.shape[0] - 1)
    if hasattr(residues, "is_cuda") and residues.is_cuda:
        f.residues_on_device = 1
        f.residues = int(residues.data_ptr())
        keep = (residues, off)
    else:
        res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint8))
        f.residues_on_device = 0
        f.residues = res.ctypes.data
        keep = (res, off)
    f.offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    return f, keep


class _DevArray:
    """Exposes a device pointer through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
            "version": 3, "strides": None, "stream": None}


class Result:
    """Owns a qp_result; arrays are numpy (host) or torch (device) views."""

    _FIELDS = {
        "pair_row_off": ("<i8", lambda r: r.n_pairs + 1),
        "row_ptr": ("<i4", lambda r: r.n_rows),
        "pair_nnz_off": ("<i8", lambda r: r.n_pairs + 1),
        "col": ("<i4", lambda r: r.nnz),
        "val": ("<f4", lambda r: r.nnz),
        "val64": ("<f8", lambda r: r.nnz),
        "dist": ("<f4", lambda r: r.k * r.k),
        "dist64": ("<f8", lambda r: r.k * r.k),
        "mea": ("<f8", lambda r: r.n_pairs),
        "log_z_hmm": ("<f8", lambda r: r.n_pairs),
        "log_z_pf": ("<f8", lambda r: r.n_pairs),
        "pair_flags": ("<i4", lambda r: r.n_pairs),
    }

    def __init__(self, ptr):
        self._ptr = ptr
        r = ptr.contents
        self.k = r.k
        self.on_device = bool(r.on_device)
        self.n_pairs = r.n_pairs
        self.n_rows = r.n_rows
        self.nnz = r.nnz
        self.kernel_ms = list(r.kernel_ms)
        self.n_fallback = r.n_fallback
        self.guard_info = list(r.guard_info)
        self.threshold_used = r.threshold_used
        self.precision = r.precision

    def array(self, name):
        r = self._ptr.contents
        typestr, n = self._FIELDS[name]
        n = int(n(r))
        addr = getattr(r, name)
        if not addr:
            return None
        shape = (self.k, self.k) if name in ("dist", "dist64") else (n,)
        if self.on_device:
            import torch
            return torch.as_tensor(_DevArray(addr, shape, typestr, self), device=f"cuda:{r.device}")
        dt = np.dtype(typestr)
        if n == 0:
            return np.zeros(shape, dtype=dt)
        buf = (ctypes.c_char * (n * dt.itemsize)).from_address(addr)
        return np.frombuffer(buf, dtype=dt, count=n).reshape(shape)

    def __getattr__(self, name):
        if name in Result._FIELDS:
            return self.array(name)
        raise AttributeError(name)

    def pair_csr(self, p: int):
        """(row_ptr, col, val, val64-or-None) of pair p as host numpy arrays."""
        def h(x):
            return x.cpu().numpy() if hasattr(x, "cpu") else x
        pro = h(self.array("pair_row_off"))
        pno = h(self.array("pair_nnz_off"))
        rp = h(self.array("row_ptr"))[pro[p]:pro[p + 1]]
        lo, hi = int(pno[p]), int(pno[p + 1])
        col = h(self.array("col"))[lo:hi]
        val = h(self.array("val"))[lo:hi]
        v64 = self.array("val64")
        v64 = h(v64)[lo:hi] if v64 is not None else None
        return rp, col, val, v64

    def free(self):
        if self._ptr is not None:
            lib().qp_result_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qp_posteriors(residues, offsets, params, out_on_device: bool = False, device: int = 0,
                  stream=None, **overrides) -> Result:
    """All-pairs posteriors, sparse matrices and MEA distances of one family.

    ``params`` is a qp_params or any object with the model fields."""
    L = lib()
    fam, keep = make_family(residues, offsets)
    prm = params if isinstance(params, qp_params) else make_params(params, device=device,
                                                                   stream=stream, **overrides)
    out = ctypes.POINTER(qp_result)()
    rc = L.qp_posteriors(ctypes.byref(fam), ctypes.byref(prm), int(bool(out_on_device)),
                         ctypes.byref(out))
    del keep
    _check(rc)
    return Result(out)


def qp_posteriors_range(residues, offsets, params, p_begin: int, p_end: int, out_on_device: bool = False,
                        device: int = 0, stream=None, **overrides) -> Result:
    """The pairs p_begin <= p < p_end of a family (qp_posteriors_range in
    qp.h): pair q of the result is pair p_begin + q of the family; distances
    are k x k with only the range's pairs filled."""
    L = lib()
    fam, keep = make_family(residues, offsets)
    prm = params if isinstance(params, qp_params) else make_params(params, device=device,
                                                                   stream=stream, **overrides)
    out = ctypes.POINTER(qp_result)()
    rc = L.qp_posteriors_range(ctypes.byref(fam), ctypes.byref(prm), int(p_begin), int(p_end),
                               int(bool(out_on_device)), ctypes.byref(out))
    del keep
    _check(rc)
    return Result(out)


def qp_split_pairs(offsets, n_parts: int) -> np.ndarray:
    """Equal-work split of a family's pairs (qp_split_pairs in qp.h; host
    only): int64 bounds[n_parts + 1], part i = pairs bounds[i] <= p <
    bounds[i+1]."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    k = int(off.shape[0] - 1)
    bounds = np.zeros(int(n_parts) + 1, dtype=np.int64)
    _check(lib().qp_split_pairs(k, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(n_parts),
                                bounds.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return bounds


QP_STATIC_MAX_LEN = 512      # the same limit as QP_STATIC_MAX_LEN in qp.h


def qp_pair_posteriors_static(residues, m: int, n: int, params, row_ptr, col, val,
                              pair_out, device: int = 0, stream=None) -> int:
    """Allocation-free single-pair call (qp_pair_posteriors_static in qp.h).

    For callers that may not allocate device memory while they run.  Every
    array is a caller-owned contiguous CUDA tensor on ``device`` (or on
    ``params.device`` when ``params`` is a qp_params): ``residues``
    uint8[m + n] (x then y, ASCII), ``row_ptr`` int32[m + 1], ``col``
    int32[cap], ``val`` float32[cap], ``pair_out`` float64[4] (MEA score,
    distance, log Z_hmm, log Z_pf).  The call runs on ``stream``, by default
    torch's current stream of that device.  Returns the number of entries
    written."""
    import torch
    dev = int(params.device) if isinstance(params, qp_params) else int(device)
    if stream is None:
        stream = torch.cuda.current_stream(torch.device("cuda", dev)).cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    if isinstance(params, qp_params):
        prm = params
        prm.stream = stream or None
    else:
        prm = make_params(params, device=dev, stream=stream)

    def need(t, name, dtype, numel):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise QpError(QP_EINVAL, f"{name} must be a CUDA tensor")
        if t.device.index != dev:
            raise QpError(QP_EINVAL, f"{name} is on cuda:{t.device.index}, the call runs on cuda:{dev}")
        if t.dtype != dtype:
            raise QpError(QP_EINVAL, f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise QpError(QP_EINVAL, f"{name} must be contiguous")
        if t.numel() < numel:
            raise QpError(QP_EINVAL, f"{name} holds {t.numel()} elements, {numel} needed")

    m, n = int(m), int(n)
    need(residues, "residues", torch.uint8, m + n)
    need(row_ptr, "row_ptr", torch.int32, m + 1)
    need(pair_out, "pair_out", torch.float64, 4)
    cap = 0
    if col is not None or val is not None:
        need(col, "col", torch.int32, 0)
        need(val, "val", torch.float32, 0)
        cap = min(int(col.numel()), int(val.numel()))
    nnz = ctypes.c_int64(0)
    rc = lib().qp_pair_posteriors_static(
        int(residues.data_ptr()), m, n, ctypes.byref(prm), int(row_ptr.data_ptr()),
        int(col.data_ptr()) if cap else None, int(val.data_ptr()) if cap else None, cap,
        int(pair_out.data_ptr()), ctypes.byref(nnz))
    _check(rc)
    return int(nnz.value)


def qp_guide_tree(dist, device: Optional[int] = None, stream=None):
    """Weighted UPGMA guide tree (qp_guide_tree in qp.h).

    ``dist`` is a k x k distance matrix (only i < j is read): a numpy array
    (host; the outputs are numpy) or a CUDA tensor (device; the outputs are
    CUDA tensors on its device, and the call runs on torch's current stream
    unless ``stream`` is given).  Returns (merges int32 (k-1, 2), heights
    float64 (k-1,)): the ids joined at step s (leaves 0..k-1, the cluster of
    step s is k + s) and half the joining distance."""
    if hasattr(dist, "is_cuda") and dist.is_cuda:
        import torch
        d = dist.to(torch.float64).contiguous()
        if d.dim() != 2 or d.shape[0] != d.shape[1]:
            raise ValueError("dist must be a square matrix")
        k = int(d.shape[0])
        dev = d.device.index if device is None else int(device)
        merges = torch.empty((max(k - 1, 0), 2), dtype=torch.int32, device=d.device)
        heights = torch.empty(max(k - 1, 0), dtype=torch.float64, device=d.device)
        if stream is None:
            stream = torch.cuda.current_stream(d.device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(lib().qp_guide_tree(int(d.data_ptr()), k, 1, dev, stream or None,
                                   int(merges.data_ptr()), int(heights.data_ptr())))
        return merges, heights
    d = np.ascontiguousarray(dist, dtype=np.float64)
    if d.ndim != 2 or d.shape[0] != d.shape[1]:
        raise ValueError("dist must be a square matrix")
    k = int(d.shape[0])
    merges = np.zeros((max(k - 1, 0), 2), dtype=np.int32)
    heights = np.zeros(max(k - 1, 0), dtype=np.float64)
    if hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(lib().qp_guide_tree(d.ctypes.data, k, 0, 0 if device is None else int(device), stream or None,
                               merges.ctypes.data, heights.ctypes.data))
    return merges, heights


def qp_consistency(posteriors: Result, offsets, merges, T: int = 200, n_max: int = 200, h: float = 3.0,
                   threshold: float = 0.01, out_on_device: bool = False) -> Result:
    """Selective consistency (qp_consistency in qp.h): the relaxed posterior
    matrices of ``posteriors`` over the guide tree ``merges`` (an int32 (k-1, 2)
    numpy array, or a CUDA tensor on the result's device)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    cp = qp_consistency_params(int(T), int(n_max), float(h), float(threshold))
    if hasattr(merges, "is_cuda") and merges.is_cuda:
        import torch
        mg = merges.to(torch.int32).contiguous()
        addr, on_dev = int(mg.data_ptr()), 1
    else:
        mg = np.ascontiguousarray(np.asarray(merges, dtype=np.int32))
        addr, on_dev = mg.ctypes.data, 0
    out = ctypes.POINTER(qp_result)()
    rc = lib().qp_consistency(posteriors._ptr, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), addr, on_dev,
                              ctypes.byref(cp), int(bool(out_on_device)), ctypes.byref(out))
    del mg
    _check(rc)
    return Result(out)


def qp_result_free(result: Result):
    result.free()


def qp_get_counter(name: str, device: int = 0) -> int:
    """Call counter of a device (qp_get_counter in qp.h)."""
    v = ctypes.c_int64(0)
    _check(lib().qp_get_counter(int(device), name.encode(), ctypes.byref(v)))
    return int(v.value)


def qp_set_option(name: str, value: int, device: int = 0):
    """Launch knob of the FP32 kernel (qp_set_option in qp.h); -1 = automatic."""
    _check(lib().qp_set_option(int(device), name.encode(), int(value)))


class Server:
    """Serving loop with continuous batching (qp_server_* in qp.h)."""

    def __init__(self, params, mem_budget: int, device: int = 0, out_on_device: bool = False):
        self._keep = params if isinstance(params, qp_params) else make_params(params, device=device)
        h = ctypes.c_void_p()
        self._h = None
        _check(lib().qp_server_create(ctypes.byref(self._keep), int(mem_budget), int(bool(out_on_device)),
                                      ctypes.byref(h)))
        self._h = h

    def stats(self) -> dict:
        st = qp_server_stats()
        _check(lib().qp_server_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in qp_server_stats._fields_}

    def submit(self, residues, offsets) -> int:
        fam, keep = make_family(residues, offsets)
        t = ctypes.c_uint64()
        rc = lib().qp_server_submit(self._h, ctypes.byref(fam), ctypes.byref(t))
        del keep
        _check(rc)
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1) -> Optional[Result]:
        out = ctypes.POINTER(qp_result)()
        rc = lib().qp_server_poll(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(out))
        if rc in (QP_ENOTREADY, QP_ETIMEOUT):
            return None
        _check(rc)
        return Result(out)

    def cancel(self, ticket: int):
        _check(lib().qp_server_cancel(self._h, ctypes.c_uint64(ticket)))

    def destroy(self):
        if self._h is not None and self._h.value:
            lib().qp_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def qp_server_create(params, mem_budget: int, device: int = 0, out_on_device: bool = False) -> Server:
    return Server(params, mem_budget, device, out_on_device)


def qp_server_submit(server: Server, residues, offsets) -> int:
    return server.submit(residues, offsets)


def qp_server_poll(server: Server, ticket: int, timeout_ms: int = -1):
    return server.poll(ticket, timeout_ms)


def qp_server_cancel(server: Server, ticket: int):
    server.cancel(ticket)


def qp_server_get_stats(server: Server) -> dict:
    return server.stats()


def qp_server_destroy(server: Server):
    server.destroy()
