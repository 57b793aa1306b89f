"""Writes tests/golden/tiny_pairs.json from the oracle alone.

Tiny seeded pairs (lengths 1-7, every model value printed in full) whose
posteriors, totals, MEA scores and distances the oracle computes; the oracle
itself is pinned by brute-force enumeration and closed forms in
tests/test_oracle_pins.py.  The fixture freezes those values so that any later
change to the oracle's arithmetic shows up, and gives the CUDA path small
cases with every cell known.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = [(1, 1), (1, 4), (4, 1), (2, 2), (3, 5), (6, 6), (7, 3)]


def main():
    rng = np.random.Generator(np.random.PCG64(20151223))
    q = synth.background()
    prm = synth.default_params(threshold=0.01)
    out = {"params": "synth.default_params(threshold=0.01)", "alphabet": synth.ALPHABET, "cases": []}
    for m, n in CASES:
        x = rng.choice(20, size=m, p=q).astype(np.uint8)
        y = rng.choice(20, size=n, p=q).astype(np.uint8)
        r = oracle.pair(x, y, prm)
        out["cases"].append({
            "x": "".join(synth.ALPHABET[c] for c in x),
            "y": "".join(synth.ALPHABET[c] for c in y),
            "P": np.asarray(r["P"]).tolist(),
            "logz_hmm": r["logz_hmm"], "logz_pf": r["logz_pf"],
            "mea": r["mea"], "dist": r["dist"],
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_pairs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
