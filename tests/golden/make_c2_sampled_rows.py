"""Writes tests/golden/c2_sampled_rows.json: the oracle's y = K x at 12 full rows of the
65,536-point three-layer workload (interfaces y = 0, -2; k = 4, 6, 8; eta = 1, 2, 3; 64
circles and ellipses of 1024 nodes, seed 12452), for a seeded dense x.  Calls only
oracle/ and workloads/ (the dense definition of Sec. 3.3, eq. matrixelmemts, with G^r
by the direct interface solve and Sommerfeld quadrature).

Rows: one seeded row per layer, five more seeded rows, and on each side of each
interface the collocation point closest to it (where the reaction part is largest
and the expansions of cells that straddle the interface matter most).

    python tests/golden/make_c2_sampled_rows.py        (a few minutes on 8 cores)
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nystrom as onys  # noqa: E402
from workloads import config_c2  # noqa: E402

SEED = 65_536


def sample(pts, interfaces):
    """x and the rows, from the seed and the geometry (numpy's PCG64: the same on every machine)."""
    n = pts.shape[0]
    rng = np.random.default_rng(SEED)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = pts[:, 1]
    lay = np.zeros(n, dtype=np.int64)
    for yi in interfaces:
        lay += (y < yi).astype(np.int64)
    rows = [int(rng.choice(np.flatnonzero(lay == l))) for l in range(len(interfaces) + 1)]
    rows += [int(r) for r in rng.choice(n, 5, replace=False)]
    for yi in interfaces:
        for side in (y > yi, y < yi):
            idx = np.flatnonzero(side)
            rows.append(int(idx[np.argmin(np.abs(y[idx] - yi))]))
    return x, np.array(rows, dtype=np.int64)


def main():
    wl = config_c2()
    pts, w, _, _ = onys.elements(wl.bodies)
    x, rows = sample(pts, wl.medium.interfaces)
    t0 = time.time()
    y = onys.dense_rows(wl.medium, pts, w, rows) @ x
    out = {
        "what": "y = K x at 12 full rows of the 65,536-point three-layer workload (k = 4, 6, 8), seeded "
                "dense x; K by the oracle's dense definition (Sec. 3.3, eq. matrixelmemts)",
        "generator": "tests/golden/make_c2_sampled_rows.py (oracle/ only)",
        "seed": SEED, "n": int(pts.shape[0]),
        "x_checksum": [float(np.sum(x).real), float(np.sum(x).imag)],
        "rows": [int(r) for r in rows],
        "y": [[float(v.real), float(v.imag)] for v in y],
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_sampled_rows.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
