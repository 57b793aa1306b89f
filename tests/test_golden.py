"""Golden fixtures (tests/golden/): written by make_golden.py from the oracle.

CPU: the oracle still reproduces them, and the 1 x 1 case matches its closed
form.  GPU: both forms of the CUDA path reproduce every cell."""
import json
import math
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    with open(os.path.join(HERE, "golden", "tiny_pairs.json")) as f:
        return json.load(f)


def test_oracle_reproduces_golden():
    import oracle
    g = _golden()
    prm = synth.default_params(threshold=0.01)
    for c in g["cases"]:
        r = oracle.pair(oracle.encode(c["x"]), oracle.encode(c["y"]), prm)
        assert np.abs(np.asarray(r["P"]) - np.asarray(c["P"])).max() <= 1e-13
        for k in ("logz_hmm", "logz_pf", "mea", "dist"):
            assert abs(r[k] - c[k]) <= 1e-12 * max(1.0, abs(c[k])), k


def test_one_by_one_case_is_the_closed_form():
    """Only the M state can emit a single residue pair: P = 1, d = 0,
    Z_hmm = pi_M p(x, y) tau_M, Z_pf = exp(s(x, y) / T)."""
    g = _golden()
    prm = synth.default_params(threshold=0.01)
    c = next(c for c in g["cases"] if len(c["x"]) == 1 and len(c["y"]) == 1)
    a, b = g["alphabet"].index(c["x"]), g["alphabet"].index(c["y"])
    assert c["P"] == [[1.0]] and c["dist"] == 0.0 and c["mea"] == 1.0
    zh = math.log(prm.pi[0]) + math.log(prm.emit_pair[a, b]) + math.log(prm.end_w[0])
    assert abs(c["logz_hmm"] - zh) <= 1e-12
    assert abs(c["logz_pf"] - prm.score[a, b] / prm.temperature) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-9)])
def test_cuda_path_reproduces_golden(precision, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1512_07437_b300 as qp
    g = _golden()
    prm = synth.default_params(threshold=1e-30)
    for c in g["cases"]:
        fam = synth.family_from_strings([c["x"], c["y"]])
        r = qp.qp_posteriors(fam.residues, fam.offsets, prm, precision=precision)
        P = np.asarray(c["P"])
        m, n = P.shape
        rp, col, val, v64 = r.pair_csr(0)
        D = np.zeros((m, n))
        v = v64 if v64 is not None else val.astype(np.float64)
        for i in range(m):
            D[i, col[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        assert np.abs(D - P).max() <= tol, (c["x"], c["y"])
        assert abs(float(r.dist64[0, 1]) - c["dist"]) <= tol
        lt = 2e-4 if precision == "f32" else 1e-9
        assert abs(float(r.log_z_hmm[0]) - c["logz_hmm"]) <= lt * max(1.0, abs(c["logz_hmm"]))
        assert abs(float(r.log_z_pf[0]) - c["logz_pf"]) <= lt * max(1.0, abs(c["logz_pf"]))
        r.free()
