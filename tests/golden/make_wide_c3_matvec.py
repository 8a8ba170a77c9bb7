"""Writes tests/golden/wide_c3_matvec.json: the oracle's y = K x for two seeded x on the
small wide-band geometry in the four-layer medium (interfaces y = 0, -6, -12; k = 6, 10,
8, 12; ten bodies of 48 nodes spread over [-40, 40] x [-18, 6], workloads.layered_wide_c3).
At leaf size 8 its tree has orders up to 63 and cells straddling the interfaces, with
column-separated reaction pairs whose effective distance is a small fraction of the cell
width.  Calls only oracle/ and workloads/ (the dense definition, Sec. 3.3 eq.
matrixelmemts).

    python tests/golden/make_wide_c3_matvec.py        (about 6 minutes on 8 cores)
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nystrom as onys  # noqa: E402
from workloads import layered_wide_c3  # noqa: E402

SEED = 4812


def sample(n):
    rng = np.random.default_rng(SEED)
    return rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2))


def main():
    wl = layered_wide_c3()
    pts, w, _, _ = onys.elements(wl.bodies)
    X = sample(pts.shape[0])
    t0 = time.time()
    K = onys.dense_matrix(wl.medium, pts, w)
    Y = K @ X
    out = {
        "what": "y = K x, two seeded x, on workloads.layered_wide_c3 (480 points, four layers k = 6, 10, 8, 12); "
                "K by the oracle's dense definition (Sec. 3.3, eq. matrixelmemts)",
        "generator": "tests/golden/make_wide_c3_matvec.py (oracle/ only)",
        "seed": SEED, "n": int(pts.shape[0]),
        "y": [[[float(v.real), float(v.imag)] for v in Y[:, c]] for c in range(2)],
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wide_c3_matvec.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
