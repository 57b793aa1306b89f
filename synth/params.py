"""Numeric model parameters (inputs to both the CUDA path and the oracle).

The paper names its models but prints none of their parameters: the pair-HMM
follows Durbin et al. and the partition function Miyazawa (Methods, stage I);
the partition function uses VTML200 with gap penalties and temperature trained
by NOMAD on BAliBASE 3 ("Other algorithmic improvements").  Neither VTML200 nor
the trained values are available, so every number below is derived from the
synthetic background ``q`` used to generate the families:

  * match emission  p(a,b) = q(a) * [(1 - s0) [a == b] + s0 q(b)],  s0 = 0.3
    (symmetric, sums to 1, marginals equal q);
  * insert emission q(a) for the X/X2 (consume x) and Y/Y2 (consume y) states;
  * short gaps delta1 = 0.02, eps1 = 2/3 (mean length 3); long gaps
    delta2 = 0.005, eps2 = 0.9;
  * start distribution = transitions out of a virtual match state,
    end weights tau_s = 1;
  * partition-function scores: integer log-odds in half-bits,
    s(a,b) = round(2 log2(p(a,b) / (q(a) q(b)))), gap open -11, gap
    extension -1 (half-bits), temperature 3.0.

Nucleotide mode (paper, Methods, "Other algorithmic improvements": the HOXD
substitution matrix and the GTR evolutionary model).  Neither table is
printed, so ``nucleotide_params`` derives both from one GTR model:

  * base frequencies pi from ``nucleotide_background`` (seeded);
  * exchangeabilities 1 for transversions and kappa = 4 for transitions
    (A<->G, C<->T); Q_ab = r_ab pi_b, scaled to one substitution per site;
  * match emission p(a,b) = pi_a P_ab(t) with P(t) = exp(Q t) at divergence
    t = 0.4 (symmetric because GTR is reversible; marginals pi);
  * insert emission pi; the same gap model as for proteins;
  * partition-function scores: half-bit log-odds of the same joint,
    s(a,b) = round(2 log2(p(a,b) / (pi_a pi_b))) (a HOXD-style matrix: high
    on the diagonal, transitions above transversions).

The tables keep the 20 x 20 layout; the nucleotide block is the top-left
4 x 4 (codes A=0, C=1, G=2, T=3), the rest is zero.

This module computes parameters only; it contains no posterior arithmetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .families import background, nucleotide_background

COMBINE = {"rms": 0, "mean": 1, "hmm": 2, "pf": 3}
PRECISION = {"f32": 0, "f64": 1}


@dataclass
class ModelParams:
    pi: np.ndarray            # [5]  start over (M, X, Y, X2, Y2)
    delta1: float
    eps1: float
    delta2: float
    eps2: float
    emit_pair: np.ndarray     # [20, 20]
    emit_bg: np.ndarray       # [20]
    end_w: np.ndarray         # [5]
    score: np.ndarray         # [20, 20]
    gap_open: float
    gap_ext: float
    temperature: float
    end_gap_mode: int = 0
    combine: str = "rms"
    threshold: float = 0.01
    precision: str = "f32"
    alphabet: str = "protein"      # "protein" (20 letters) or "nucleotide" (ACGT)

    def replace(self, **kw) -> "ModelParams":
        d = dict(self.__dict__)
        d.update(kw)
        for key in ("pi", "emit_pair", "emit_bg", "end_w", "score"):
            d[key] = np.array(d[key], dtype=np.float64, copy=True)
        return ModelParams(**d)


def default_params(q: np.ndarray | None = None, s0: float = 0.3,
                   delta1: float = 0.02, eps1: float = 2.0 / 3.0,
                   delta2: float = 0.005, eps2: float = 0.9,
                   gap_open: float = -11.0, gap_ext: float = -1.0,
                   temperature: float = 3.0, threshold: float = 0.01,
                   combine: str = "rms", precision: str = "f32") -> ModelParams:
    q = background() if q is None else np.asarray(q, dtype=np.float64)
    eye = np.eye(20)
    p = q[:, None] * ((1.0 - s0) * eye + s0 * q[None, :])
    p = 0.5 * (p + p.T)
    tmm = 1.0 - 2.0 * delta1 - 2.0 * delta2
    pi = np.array([tmm, delta1, delta1, delta2, delta2], dtype=np.float64)
    odds = p / (q[:, None] * q[None, :])
    score = np.round(2.0 * np.log2(odds))
    return ModelParams(pi=pi, delta1=delta1, eps1=eps1, delta2=delta2, eps2=eps2,
                       emit_pair=p, emit_bg=q.copy(), end_w=np.ones(5),
                       score=score, gap_open=gap_open, gap_ext=gap_ext,
                       temperature=temperature, combine=combine,
                       threshold=threshold, precision=precision)


def gtr_joint(pi: np.ndarray, exch: np.ndarray, t: float) -> np.ndarray:
    """Joint distribution p(a,b) = pi_a P_ab(t) of a reversible GTR model with
    base frequencies pi and symmetric exchangeabilities exch (zero diagonal),
    its rate matrix scaled to one expected substitution per site."""
    pi = np.asarray(pi, dtype=np.float64)
    Q = exch * pi[None, :]
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    Q /= -(pi * np.diag(Q)).sum()
    # symmetric form D^1/2 Q D^-1/2 for a stable exponential
    d = np.sqrt(pi)
    S = d[:, None] * Q / d[None, :]
    S = 0.5 * (S + S.T)
    w, V = np.linalg.eigh(S)
    P = (V * np.exp(w * t)) @ V.T
    P = P / d[:, None] * d[None, :]
    J = pi[:, None] * P
    J = 0.5 * (J + J.T)
    return J / J.sum()


def nucleotide_params(pi: np.ndarray | None = None, kappa: float = 4.0, t: float = 0.4,
                      delta1: float = 0.02, eps1: float = 2.0 / 3.0,
                      delta2: float = 0.005, eps2: float = 0.9,
                      gap_open: float = -11.0, gap_ext: float = -1.0,
                      temperature: float = 3.0, threshold: float = 0.01,
                      combine: str = "rms", precision: str = "f32") -> ModelParams:
    pi = nucleotide_background() if pi is None else np.asarray(pi, dtype=np.float64)
    exch = np.ones((4, 4))
    exch[0, 2] = exch[2, 0] = kappa          # A <-> G
    exch[1, 3] = exch[3, 1] = kappa          # C <-> T
    J = gtr_joint(pi, exch, t)
    p = np.zeros((20, 20))
    p[:4, :4] = J
    q = np.zeros(20)
    q[:4] = pi
    score = np.zeros((20, 20))
    score[:4, :4] = np.round(2.0 * np.log2(J / (pi[:, None] * pi[None, :])))
    tmm = 1.0 - 2.0 * delta1 - 2.0 * delta2
    start = np.array([tmm, delta1, delta1, delta2, delta2], dtype=np.float64)
    return ModelParams(pi=start, delta1=delta1, eps1=eps1, delta2=delta2, eps2=eps2,
                       emit_pair=p, emit_bg=q, end_w=np.ones(5), score=score,
                       gap_open=gap_open, gap_ext=gap_ext, temperature=temperature,
                       combine=combine, threshold=threshold, precision=precision,
                       alphabet="nucleotide")
