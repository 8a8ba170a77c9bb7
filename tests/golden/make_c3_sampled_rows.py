"""Writes tests/golden/c3_sampled_rows.json: the oracle's y = K x at sampled rows of the
largest workload (C3: N = 1,048,576, four layers), for an x that is non-zero on a seeded
subset of 4096 columns.  Calls only oracle/ and workloads/ (the dense definition, Sec. 3.3
eq. matrixelmemts, with G^r by the direct interface solve and Sommerfeld quadrature).

The full rows of this matrix are out of reach of the oracle in a test (a million Sommerfeld
integrals per row), so the columns are a seeded 4k-point subset, as the precision form's
configuration asks; the GPU side multiplies the same sparse x at full size.

    python tests/golden/make_c3_sampled_rows.py        (about 5 minutes on 8 cores)
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nystrom as onys  # noqa: E402
from workloads import config_c3  # noqa: E402

SEED = 31_2024
N_COLS = 4096
N_ROWS = 64
N_ROWS_IN_COLS = 8   # rows whose own column is in the subset (self terms)
# the oracle's quadrature tolerance, tightest first: for a few far pairs (|x - x'| ~ 70, the
# detour h = 1/|x - x'| close under the guided-mode poles) the adaptive rule's error
# estimate does not reach 1e-13 within its subdivision cap, although the values agree
# with a 10x larger cap to 6e-14; such a row is recomputed at the next tolerance
TOLS = (1e-12, 1e-11, 1e-10)


def row_value(med, pts, w, r, cols, x):
    for tol in TOLS:
        try:
            return onys.dense_row_block(med, pts, w, int(r), cols, tol_rel=tol) @ x, tol
        except RuntimeError:
            continue
    raise RuntimeError(f"row {r}: the oracle quadrature did not converge at {TOLS[-1]}")


def sample(n):
    """Columns, x on them, and rows, from the seed (numpy's PCG64: the same on every machine)."""
    rng = np.random.default_rng(SEED)
    cols = np.sort(rng.choice(n, N_COLS, replace=False))
    x = rng.standard_normal(N_COLS) + 1j * rng.standard_normal(N_COLS)
    rows_in = rng.choice(cols, N_ROWS_IN_COLS, replace=False)
    rows_out = rng.choice(np.setdiff1d(np.arange(n), cols), N_ROWS - N_ROWS_IN_COLS, replace=False)
    rows = np.concatenate([rows_in, rows_out])
    return cols, x, rows


def main():
    wl = config_c3()
    pts, w, _, _ = onys.elements(wl.bodies)
    cols, x, rows = sample(pts.shape[0])
    t0 = time.time()
    res = [row_value(wl.medium, pts, w, r, cols, x) for r in rows]
    y = np.array([v for v, _ in res])
    out = {
        "what": "y = K x at sampled rows of C3 (N = 1,048,576, 4 layers, k = 6, 10, 8, 12), x non-zero on "
                "4096 seeded columns; K by the oracle's dense definition (Sec. 3.3, eq. matrixelmemts)",
        "generator": "tests/golden/make_c3_sampled_rows.py (oracle/ only)",
        "seed": SEED, "n": int(pts.shape[0]), "n_cols": N_COLS,
        "tol_rel": [t for _, t in res],
        "x_checksum": [float(np.sum(x).real), float(np.sum(x).imag), int(np.sum(cols))],
        "rows": [int(r) for r in rows],
        "y": [[float(v.real), float(v.imag)] for v in y],
        "oracle_seconds": round(time.time() - t0, 1),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_sampled_rows.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
