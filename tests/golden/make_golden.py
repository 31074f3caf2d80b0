"""Writes tests/golden/tiny_sketches.json from the exact-Fraction brute force in
oracle/bruteforce.py (it calls nothing outside oracle/).  The paper prints no worked hash
values, so these fixtures record the definition's output on small explicit sets: element
indices and fp32 weights (as exact hex floats), k, seed, the box used, and the minhash keys
of every bucket whose box minimum is the global minimum.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import bruteforce as bf  # noqa: E402

CASES = [
    # (indices, weights, k, seed)
    ([5], [1.0], 1, 1),
    ([7, 11], [0.75, 0.25], 2, 1),               # t = 4: 4 * 0.75 = 3 = 2^2 - 1 (region edge)
    ([1, 2, 3], [0.5, 0.125, 0.375], 3, 42),
    ([100, 200, 300, 400], [0.01, 0.02, 0.03, 0.04], 5, 7),
    ([3, 9], [2.5, 0.001953125], 8, 123456789),
    ([0, 4294967295], [0.3, 0.7], 4, 2 ** 63 + 5),
    ([17], [0.0625], 6, 99),
]


def box_for(w, k, t):
    l1 = float(np.asarray(w, dtype=np.float64).sum())
    y = max(float(x) * t for x in w)
    nu_box = 0
    while 2 ** (nu_box + 1) - 1 <= y:
        nu_box += 1
    R = 14.0 * k / (t * l1)
    rho_box = 0
    while 2 ** (rho_box + 1) - 1 < R:
        rho_box += 1
    return nu_box, rho_box


def main():
    T = oracle.poisson_thresholds()
    out = []
    for idx, w, k, seed in CASES:
        w32 = np.array(w, dtype=np.float32)
        t = oracle.t_of_k(k)
        nu_box, rho_box = box_for(w32, k, t)
        keys = bf.sketch(np.array(idx, dtype=np.uint32), w32, k, t, seed, nu_box, rho_box, T)
        out.append(dict(indices=idx, weights_hex=[float(x).hex() for x in w32], k=k, t=t, seed=seed,
                        nu_box=nu_box, rho_box=rho_box,
                        keys=[None if v is None else f"{v:016x}" for v in keys]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_sketches.json")
    with open(path, "w") as f:
        json.dump(dict(source="oracle/bruteforce.py via tests/golden/make_golden.py", cases=out), f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
