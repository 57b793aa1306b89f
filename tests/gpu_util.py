"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle

TOL_F32 = 1e-5      # posterior and distance tolerance of the FP32 scaled form
TOL_F64 = 1e-9      # tolerance of the FP64 plain form
TOL_LOGZ32 = 2e-4   # log totals of the FP32 form, relative (rounding over ~10^3 steps)
TOL_LOGZ64 = 1e-9


def host(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def dense_of(res, p, m, n):
    """Dense P of pair p from the result's CSR (absent entries are 0)."""
    rp, col, val, v64 = res.pair_csr(p)
    assert rp.shape == (m + 1,)
    assert rp[0] == 0 and (np.diff(rp) >= 0).all()
    v = v64 if v64 is not None else val.astype(np.float64)
    D = np.zeros((m, n))
    for i in range(m):
        c = col[rp[i]:rp[i + 1]]
        assert (np.diff(c) > 0).all(), "columns must ascend within a row"
        assert c.size == 0 or (c.min() >= 0 and c.max() < n)
        D[i, c] = v[rp[i]:rp[i + 1]]
    return D


def compare_pair(res, fam, p, a, b, prm, tol, tol_logz, dense=True, theta=None, ref=None):
    """Error figures of one pair; asserts the bar."""
    if ref is None:
        ref = oracle.pair(fam.codes(a), fam.codes(b), prm)
    P = ref["P"]
    m, n = P.shape
    D = dense_of(res, p, m, n)
    out = {}
    if dense:
        err = np.abs(D - P).max()
        out["p_err"] = float(err)
        assert err <= tol, f"pair {p} ({a},{b}) m={m} n={n}: max |dP| = {err:.3e}"
    else:
        th = prm.threshold if theta is None else theta
        kept_ref = P >= th
        kept_gpu = D > 0
        guard = np.abs(P - th) > 1e-5
        mism = (kept_ref != kept_gpu) & guard
        assert not mism.any(), f"pair {p}: {int(mism.sum())} pattern mismatches outside the guard band"
        both = kept_ref & kept_gpu
        err = float(np.abs(D[both] - P[both]).max()) if both.any() else 0.0
        out["p_err"] = err
        out["nnz"] = int(kept_gpu.sum())
        assert err <= tol, f"pair {p}: max |dP| on kept entries = {err:.3e}"
    mea = float(host(res.mea)[p])
    dist = host(res.dist64)
    d_err = abs(float(dist[a, b]) - ref["dist"])
    out["d_err"] = d_err
    assert d_err <= tol, f"pair {p}: |d dist| = {d_err:.3e}"
    assert float(dist[b, a]) == float(dist[a, b])
    assert abs(mea - ref["mea"]) <= tol * min(m, n), f"pair {p}: MEA {mea} vs {ref['mea']}"
    lzh = host(res.log_z_hmm)
    lzp = host(res.log_z_pf)
    assert abs(lzh[p] - ref["logz_hmm"]) <= tol_logz * max(1.0, abs(ref["logz_hmm"])), \
        f"pair {p}: log Z_hmm {lzh[p]} vs {ref['logz_hmm']}"
    assert abs(lzp[p] - ref["logz_pf"]) <= tol_logz * max(1.0, abs(ref["logz_pf"])), \
        f"pair {p}: log Z_pf {lzp[p]} vs {ref['logz_pf']}"
    return out


def guard_report(res):
    """Histogram of FP32 range-guard reasons over the result's pairs."""
    from paper_1512_07437_b300 import GUARD_BITS
    fl = host(res.pair_flags)
    out = {}
    for bit, name in GUARD_BITS.items():
        c = int(((fl >> bit) & 1).sum())
        if c:
            out[name] = c
    return out
