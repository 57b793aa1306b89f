"""Seeded synthetic protein and nucleotide families.

The paper evaluates on curated benchmark families (BAliBASE, PREFAB, OXBench,
SABmark, BaliFam with ~934 sequences per set, HomFam^1K with ~1093 per family;
Methods, "Accuracy assessment").  None of those datasets is used here: every
family is generated from a seeded evolution model whose sizes, lengths and
divergences stand in for those workloads.

Evolution model (the same for every configuration):
  * a root sequence of i.i.d. residues drawn from the background ``q``;
  * substitution at rate ``s`` per site: a chosen site is replaced by a draw
    from ``q`` conditioned on differing from the current residue, so ``s`` is
    the expected changed fraction;
  * indel events start at each site with probability ``r = 0.05 * s / 0.3``;
    half are insertions, half deletions; event lengths are geometric on
    {1, 2, ...} with mean 3; inserted residues are drawn from ``q``.

Nucleotide families (alphabet ACGT) use the same model over a 4-letter
background (``nucleotide_background``); protein families are unchanged by it.

Randomness comes from ``numpy.random.Generator(PCG64(seed))`` only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

ALPHABET = "ACDEFGHIKLMNPQRSTVWY"
NUCLEOTIDES = "ACGT"
_ALPHA_BYTES = np.frombuffer(ALPHABET.encode("ascii"), dtype=np.uint8)
_NUC_BYTES = np.frombuffer(NUCLEOTIDES.encode("ascii"), dtype=np.uint8)
LETTERS = {"protein": _ALPHA_BYTES, "nucleotide": _NUC_BYTES}

# Per-configuration defaults.  The sizes follow the five workload
# configurations of the posterior stage (8 / 64 / 500 / serving / 100
# sequences).
CONFIGS = {
    "c1": dict(k=8, root=(100, 150), s=0.30, layout="star", keep=None),
    "c2": dict(k=64, root=(200, 400), s=0.40, layout="star", keep=(200, 400)),
    "c3": dict(k=500, root=(600, 600), s=(0.05, 0.25), layout="tree",
               trim=(150, 500)),
    "c4": dict(n_families=200, rate_hz=20.0, k=(10, 1000), root=(50, 1000),
               s=(0.05, 0.25), layout="tree", keep=(50, 1000)),
    "c5": dict(k=100, domains=3, domain_len=(700, 1300), p_drop=0.2,
               s=0.30, layout="star", keep=(2000, 4000)),
}


@dataclass
class Family:
    """A set of sequences laid out as one byte buffer plus offsets.

    ``residues`` holds the concatenated ASCII letters (uint8); sequence ``a``
    is ``residues[offsets[a]:offsets[a+1]]``.
    """
    residues: np.ndarray          # uint8, ASCII letters
    offsets: np.ndarray           # int64, k+1
    name: str = ""
    meta: dict = field(default_factory=dict)
    alphabet: str = "protein"     # "protein" (20 letters) or "nucleotide" (ACGT)

    @property
    def k(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def seq(self, a: int) -> str:
        return self.residues[self.offsets[a]:self.offsets[a + 1]].tobytes().decode("ascii")

    def codes(self, a: int) -> np.ndarray:
        """Residue codes of sequence ``a``: 0..19 (index into ``ALPHABET``),
        or 0..3 (index into ``NUCLEOTIDES``, U read as T)."""
        letters = LETTERS[self.alphabet]
        lut = np.full(256, 255, dtype=np.uint8)
        lut[letters] = np.arange(letters.size, dtype=np.uint8)
        if self.alphabet == "nucleotide":
            lut[ord("U")] = 3
        return lut[self.residues[self.offsets[a]:self.offsets[a + 1]]]

    def pairs(self):
        """Pairs (a, b), a < b, in the linear order p = a*k - a(a+1)/2 + (b-a-1)."""
        k = self.k
        for a in range(k):
            for b in range(a + 1, k):
                yield a, b

    @property
    def n_pairs(self) -> int:
        return self.k * (self.k - 1) // 2

    def cells(self) -> int:
        """Sum over pairs of m*n (the cell count used by the GCUPS metric)."""
        L = self.lengths.astype(np.float64)
        s = L.sum()
        return int(round((s * s - (L * L).sum()) / 2.0))


def pair_index(a: int, b: int, k: int) -> int:
    return a * k - a * (a + 1) // 2 + (b - a - 1)


def background(seed: int = 20151223) -> np.ndarray:
    """Background residue frequencies q: one seeded Dirichlet(5) draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.dirichlet(np.full(20, 5.0))
    return q / q.sum()


def nucleotide_background(seed: int = 20151224) -> np.ndarray:
    """Background nucleotide frequencies (A, C, G, T): one seeded Dirichlet(20) draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.dirichlet(np.full(4, 20.0))
    return q / q.sum()


def _background(alphabet: str) -> np.ndarray:
    return background() if alphabet == "protein" else nucleotide_background()


def _draw_residues(rng, q, n):
    return rng.choice(len(q), size=n, p=q).astype(np.uint8)


def evolve(rng, seq: np.ndarray, s: float, q: np.ndarray) -> np.ndarray:
    """One branch of the evolution model applied to a code array."""
    out = seq.copy()
    L = out.shape[0]
    if L:
        mask = rng.random(L) < s
        idx = np.nonzero(mask)[0]
        if idx.size:
            new = _draw_residues(rng, q, idx.size)
            same = new == out[idx]
            while same.any():
                new[same] = _draw_residues(rng, q, int(same.sum()))
                same = new == out[idx]
            out[idx] = new
    r = 0.05 * s / 0.3
    if L == 0:
        return out
    starts = np.nonzero(rng.random(L) < r)[0]
    if starts.size == 0:
        return out
    kinds = rng.random(starts.size) < 0.5        # True: insertion
    lens = rng.geometric(1.0 / 3.0, size=starts.size)
    pieces = []
    pos = 0
    for st, ins, ln in zip(starts.tolist(), kinds.tolist(), lens.tolist()):
        if st < pos:          # inside a region already deleted
            continue
        if ins:
            pieces.append(out[pos:st + 1])
            pieces.append(_draw_residues(rng, q, ln))
            pos = st + 1
        else:
            pieces.append(out[pos:st])
            pos = min(L, st + ln)
    pieces.append(out[pos:])
    return np.concatenate(pieces).astype(np.uint8)


def _pack(seqs: Sequence[np.ndarray], name: str, meta: dict, alphabet: str = "protein") -> Family:
    offs = np.zeros(len(seqs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in seqs])
    codes = np.concatenate(list(seqs)).astype(np.uint8)
    return Family(residues=LETTERS[alphabet][codes].copy(), offsets=offs,
                  name=name, meta=meta, alphabet=alphabet)


def family_from_strings(seqs: Sequence[str], name: str = "custom", alphabet: str = "protein") -> Family:
    """Family from Python strings (letters are not validated here)."""
    offs = np.zeros(len(seqs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in seqs])
    buf = np.frombuffer("".join(seqs).encode("ascii"), dtype=np.uint8).copy()
    return Family(residues=buf, offsets=offs, name=name, meta={}, alphabet=alphabet)


def star_family(seed: int, k: int, root_len: tuple, s: float,
                keep: Optional[tuple] = None, q=None, name="star", alphabet: str = "protein") -> Family:
    """k leaves evolved independently from one root (a star tree)."""
    q = _background(alphabet) if q is None else q
    rng = np.random.Generator(np.random.PCG64(seed))
    L0 = int(rng.integers(root_len[0], root_len[1] + 1))
    root = _draw_residues(rng, q, L0)
    seqs = []
    for _ in range(k):
        for _try in range(1000):
            leaf = evolve(rng, root, s, q)
            if leaf.size >= 1 and (keep is None or keep[0] <= leaf.size <= keep[1]):
                break
        else:
            raise RuntimeError("could not draw a leaf inside the length window")
        seqs.append(leaf)
    return _pack(seqs, name, dict(seed=seed, k=k, root_len=L0, s=s), alphabet)


def _random_tree(rng, n_leaves: int):
    """Random binary tree by repeated random joins; returns (parent, n_nodes).

    Leaves are nodes 0..n-1, internal nodes n..2n-2, root 2n-2.
    """
    active = list(range(n_leaves))
    parent = np.full(2 * n_leaves - 1, -1, dtype=np.int64)
    nxt = n_leaves
    while len(active) > 1:
        i, j = rng.choice(len(active), size=2, replace=False)
        a, b = active[i], active[j]
        parent[a] = nxt
        parent[b] = nxt
        for idx in sorted((i, j), reverse=True):
            active.pop(idx)
        active.append(nxt)
        nxt += 1
    return parent, nxt


def random_guide_tree(seed: int, k: int) -> np.ndarray:
    """A seeded random join sequence over k leaves, in the guide-tree layout
    (row s joins two ids; leaves 0..k-1, the node of step s is k + s): an
    input for stages that consume a guide tree."""
    rng = np.random.Generator(np.random.PCG64(seed))
    slots = list(range(k))
    merges = np.zeros((max(k - 1, 0), 2), dtype=np.int32)
    for s in range(k - 1):
        i, j = sorted(rng.choice(len(slots), size=2, replace=False).tolist())
        merges[s] = (slots[i], slots[j])
        slots.pop(j)
        slots[i] = k + s
    return merges


def tree_family(seed: int, k: int, root_len: tuple, s_range: tuple,
                trim: Optional[tuple] = None, keep: Optional[tuple] = None,
                q=None, name="tree", alphabet: str = "protein") -> Family:
    """k leaves evolved down a seeded random binary tree.

    Every branch draws its own substitution rate from U[s_range].  With
    ``trim`` each leaf is cut to a random window of length U[trim] (when it is
    longer).  With ``keep`` a leaf shorter than keep[0] is re-evolved from its
    parent (bounded tries) and a longer one is cut to a random window.
    """
    q = _background(alphabet) if q is None else q
    rng = np.random.Generator(np.random.PCG64(seed))
    parent, n_nodes = _random_tree(rng, k)
    L0 = int(rng.integers(root_len[0], root_len[1] + 1))
    seqs = [None] * n_nodes
    root = n_nodes - 1
    seqs[root] = _draw_residues(rng, q, L0)
    children = [[] for _ in range(n_nodes)]
    for v in range(n_nodes - 1):
        children[int(parent[v])].append(v)
    stack = [root]
    order = []
    while stack:
        v = stack.pop()
        order.append(v)
        stack.extend(children[v])
    bs = {}
    for v in order:
        if v == root:
            continue
        s = float(rng.uniform(s_range[0], s_range[1]))
        bs[v] = s
        seqs[v] = evolve(rng, seqs[int(parent[v])], s, q)
    leaves = []
    for v in range(k):
        x = seqs[v]
        if keep is not None:
            tries = 0
            while x.size < keep[0] and tries < 50:
                x = evolve(rng, seqs[int(parent[v])], bs[v], q)
                tries += 1
            if x.size < 1:
                x = _draw_residues(rng, q, 1)
            if x.size > keep[1]:
                st = int(rng.integers(0, x.size - keep[1] + 1))
                x = x[st:st + keep[1]]
        if trim is not None:
            tgt = int(rng.integers(trim[0], trim[1] + 1))
            if x.size > tgt:
                st = int(rng.integers(0, x.size - tgt + 1))
                x = x[st:st + tgt]
        if x.size < 1:
            x = _draw_residues(rng, q, 1)
        leaves.append(x)
    return _pack(leaves, name, dict(seed=seed, k=k, root_len=L0), alphabet)


def domain_family(seed: int, k: int, n_domains: int, domain_len: tuple,
                  p_drop: float, s: float, keep: tuple, q=None,
                  name="domains") -> Family:
    """Long multidomain-like members: concatenated seeded domain roots, each
    member dropping each domain with probability p_drop (at least one kept),
    then evolved on a star tree; members outside ``keep`` are redrawn."""
    q = background() if q is None else q
    rng = np.random.Generator(np.random.PCG64(seed))
    doms = [_draw_residues(rng, q, int(rng.integers(domain_len[0], domain_len[1] + 1)))
            for _ in range(n_domains)]
    seqs = []
    for _ in range(k):
        for _try in range(10000):
            kept = rng.random(n_domains) >= p_drop
            if not kept.any():
                kept[int(rng.integers(0, n_domains))] = True
            root = np.concatenate([d for d, kk in zip(doms, kept) if kk])
            leaf = evolve(rng, root, s, q)
            if keep[0] <= leaf.size <= keep[1]:
                break
        else:
            raise RuntimeError("could not draw a member inside the length window")
        seqs.append(leaf)
    return _pack(seqs, name, dict(seed=seed, k=k))


def make_family(config: str, seed: int = 1) -> Family:
    """The family of configuration ``config`` ("c1", "c2", "c3", "c5")."""
    c = CONFIGS[config]
    if config in ("c1", "c2"):
        return star_family(seed, c["k"], c["root"], c["s"], keep=c.get("keep"),
                           name=config)
    if config == "c3":
        return tree_family(seed, c["k"], c["root"], c["s"], trim=c["trim"],
                           name=config)
    if config == "c5":
        return domain_family(seed, c["k"], c["domains"], c["domain_len"],
                             c["p_drop"], c["s"], c["keep"], name=config)
    raise KeyError(config)


def make_serving_trace(seed: int = 4, n_families: Optional[int] = None,
                       rate_hz: Optional[float] = None,
                       k_range: Optional[tuple] = None,
                       len_range: Optional[tuple] = None):
    """Serving workload: families arriving as a Poisson process.

    Returns a list of (arrival_time_s, Family).  Family sizes are
    log-uniform over ``k_range``; each family's root length is U[len_range]
    and its members are evolved down a random tree, kept within len_range.
    """
    c = CONFIGS["c4"]
    n_families = c["n_families"] if n_families is None else n_families
    rate_hz = c["rate_hz"] if rate_hz is None else rate_hz
    k_range = c["k"] if k_range is None else k_range
    len_range = c["root"] if len_range is None else len_range
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for f in range(n_families):
        t += float(rng.exponential(1.0 / rate_hz))
        k = int(round(math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1])))))
        k = max(2, k)
        fam_seed = int(rng.integers(0, 2**31 - 1))
        fam = tree_family(fam_seed, k, len_range, c["s"], keep=len_range,
                          name=f"c4-{f}")
        out.append((t, fam))
    return out
