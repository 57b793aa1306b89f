"""Brute-force enumerators for tiny pairs (test helpers, pure Python).

They sum over every explicit path / alignment / matching instead of running
any dynamic programme, so they check the oracle's recurrences from outside.
Model (the reading the repository documents): a 5-state pair-HMM
(M, X, Y, X2, Y2; M emits a pair, X/X2 consume x, Y/Y2 consume y; no
X<->Y, X<->X2 or Y<->Y2 moves) and a 3-state partition function over
alignments whose gap runs in x and in y never touch.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

M, X, Y, X2, Y2 = range(5)
DI = {M: 1, X: 1, X2: 1, Y: 0, Y2: 0}
DJ = {M: 1, X: 0, X2: 0, Y: 1, Y2: 1}


def _trans(prm):
    t = np.zeros((5, 5))
    d1, e1, d2, e2 = prm.delta1, prm.eps1, prm.delta2, prm.eps2
    t[M, M] = 1 - 2 * d1 - 2 * d2
    t[M, X] = t[M, Y] = d1
    t[M, X2] = t[M, Y2] = d2
    t[X, X] = t[Y, Y] = e1
    t[X, M] = t[Y, M] = 1 - e1
    t[X2, X2] = t[Y2, Y2] = e2
    t[X2, M] = t[Y2, M] = 1 - e2
    return t


def hmm_paths(x, y, prm):
    """Yield (probability, list of (state, i, j)) for every state path that
    emits all of x and y (1-based i, j of the emitted residues)."""
    m, n = len(x), len(y)
    t = _trans(prm)
    p, q, pi, tau = prm.emit_pair, prm.emit_bg, prm.pi, prm.end_w

    def emit(s, i, j):
        if s == M:
            return p[x[i - 1], y[j - 1]]
        if s in (X, X2):
            return q[x[i - 1]]
        return q[y[j - 1]]

    def rec(i, j, s, prob, path):
        if i == m and j == n:
            yield prob * tau[s], path
            return
        for r in range(5):
            if t[s, r] == 0.0:
                continue
            ni, nj = i + DI[r], j + DJ[r]
            if ni > m or nj > n:
                continue
            yield from rec(ni, nj, r, prob * t[s, r] * emit(r, ni, nj), path + [(r, ni, nj)])

    for s in range(5):
        if pi[s] == 0.0:
            continue
        i, j = DI[s], DJ[s]
        if i > m or j > n:
            continue
        yield from rec(i, j, s, pi[s] * emit(s, i, j), [(s, i, j)])


def hmm_brute(x, y, prm):
    """Z, match posterior P[i-1, j-1], gap posteriors per row / column."""
    m, n = len(x), len(y)
    Z = 0.0
    PM = np.zeros((m, n))
    GX = np.zeros(m)
    GY = np.zeros(n)
    for prob, path in hmm_paths(x, y, prm):
        Z += prob
        for s, i, j in path:
            if s == M:
                PM[i - 1, j - 1] += prob
            elif s in (X, X2):
                GX[i - 1] += prob
            else:
                GY[j - 1] += prob
    return Z, PM / Z, GX / Z, GY / Z


def alignments(m, n):
    """All alignments as op strings over {M, E (x_i vs gap), F (gap vs y_j)}
    in which an E run is never directly next to an F run."""
    out = []

    def rec(i, j, last, ops):
        if i == m and j == n:
            out.append(ops)
            return
        if i < m and j < n:
            rec(i + 1, j + 1, "M", ops + "M")
        if i < m and last != "F":
            rec(i + 1, j, "E", ops + "E")
        if j < n and last != "E":
            rec(i, j + 1, "F", ops + "F")

    rec(0, 0, "", "")
    return out


def pf_weight(ops, x, y, prm):
    """Boltzmann weight exp(score / T) of one alignment (affine gaps)."""
    T = prm.temperature
    i = j = 0
    s = 0.0
    prev = ""
    for o in ops:
        if o == "M":
            s += prm.score[x[i], y[j]]
            i += 1
            j += 1
        elif o == "E":
            s += prm.gap_ext if prev == "E" else prm.gap_open
            i += 1
        else:
            s += prm.gap_ext if prev == "F" else prm.gap_open
            j += 1
        prev = o
    return math.exp(s / T)


def aligned_pairs(ops):
    i = j = 0
    res = []
    for o in ops:
        if o == "M":
            i += 1
            j += 1
            res.append((i, j))
        elif o == "E":
            i += 1
        else:
            j += 1
    return res


def pf_brute(x, y, prm):
    m, n = len(x), len(y)
    Z = 0.0
    PP = np.zeros((m, n))
    GX = np.zeros(m)
    GY = np.zeros(n)
    for ops in alignments(m, n):
        w = pf_weight(ops, x, y, prm)
        Z += w
        i = j = 0
        for o in ops:
            if o == "M":
                i += 1
                j += 1
                PP[i - 1, j - 1] += w
            elif o == "E":
                i += 1
                GX[i - 1] += w
            else:
                j += 1
                GY[j - 1] += w
    return Z, PP / Z, GX / Z, GY / Z


def mea_brute(P):
    """Largest sum of P over index sets strictly increasing in both axes."""
    m, n = P.shape
    best = 0.0
    for r in range(1, min(m, n) + 1):
        for rows in itertools.combinations(range(m), r):
            for cols in itertools.combinations(range(n), r):
                s = sum(P[a, b] for a, b in zip(rows, cols))
                if s > best:
                    best = s
    return best


def gotoh(x, y, prm):
    """Best-scoring alignment under the same affine scheme and the same
    no-adjacent-opposite-gaps rule (max-plus dynamic programme with
    traceback).  Returns (score, set of aligned (i, j), 1-based)."""
    m, n = len(x), len(y)
    NEG = -1e300
    S = prm.score
    go, ge = prm.gap_open, prm.gap_ext
    VM = np.full((m + 1, n + 1), NEG)
    VE = np.full((m + 1, n + 1), NEG)
    VF = np.full((m + 1, n + 1), NEG)
    VM[0, 0] = 0.0
    for i in range(m + 1):
        for j in range(n + 1):
            if i == 0 and j == 0:
                continue
            if i and j:
                VM[i, j] = S[x[i - 1], y[j - 1]] + max(VM[i - 1, j - 1], VE[i - 1, j - 1], VF[i - 1, j - 1])
            if i:
                VE[i, j] = max(VM[i - 1, j] + go, VE[i - 1, j] + ge)
            if j:
                VF[i, j] = max(VM[i, j - 1] + go, VF[i, j - 1] + ge)
    # traceback
    i, j = m, n
    st = int(np.argmax([VM[m, n], VE[m, n], VF[m, n]]))
    best = max(VM[m, n], VE[m, n], VF[m, n])
    pairs = set()
    while i > 0 or j > 0:
        if st == 0:
            pairs.add((i, j))
            prev = [VM[i - 1, j - 1], VE[i - 1, j - 1], VF[i - 1, j - 1]]
            st = int(np.argmax(prev))
            i -= 1
            j -= 1
        elif st == 1:
            st = 0 if VM[i - 1, j] + go >= VE[i - 1, j] + ge else 1
            i -= 1
        else:
            st = 0 if VM[i, j - 1] + go >= VF[i, j - 1] + ge else 2
            j -= 1
    return best, pairs
