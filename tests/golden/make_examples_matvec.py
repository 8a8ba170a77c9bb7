"""Writes tests/golden/examples_matvec.json: the oracle's y = K x for a seeded x on small
discretisations of the paper's three numerical examples (Sec. 5): Example 1, the L-shape across
five layers (300 elements); Example 2, two 'peanut' scatterers in six layers (2 x 120); Example 3,
five 'flower' scatterers in six layers (5 x 60).  Media, shapes and positions are those of
workloads.example1/2/3.  Calls only oracle/ and workloads/ (the dense definition, Sec. 3.3 eq.
matrixelmemts).

    python tests/golden/make_examples_matvec.py        (several minutes on 8 cores)
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nystrom as onys  # noqa: E402
from workloads import example1, example2, example3  # noqa: E402

CASES = {"E1": (example1, 300), "E2": (example2, 240), "E3": (example3, 300)}
SEED = 5_2025


def sample(n, name):
    rng = np.random.default_rng([SEED, sorted(CASES).index(name)])
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def main():
    out = {"what": "y = K x, seeded x, on small discretisations of Examples 1-3 (Sec. 5); K by the oracle's "
                   "dense definition (Sec. 3.3, eq. matrixelmemts)",
           "generator": "tests/golden/make_examples_matvec.py (oracle/ only)", "seed": SEED, "cases": {}}
    for name, (make, n) in CASES.items():
        wl = make(n)
        pts, w, _, _ = onys.elements(wl.bodies)
        x = sample(pts.shape[0], name)
        t0 = time.time()
        y = onys.dense_matrix(wl.medium, pts, w) @ x
        out["cases"][name] = {"n": int(pts.shape[0]), "y": [[float(v.real), float(v.imag)] for v in y],
                              "oracle_seconds": round(time.time() - t0, 1)}
        print(name, pts.shape[0], out["cases"][name]["oracle_seconds"], "s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "examples_matvec.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path)


if __name__ == "__main__":
    main()
