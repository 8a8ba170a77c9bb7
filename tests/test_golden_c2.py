"""The stored C2 sampled rows (tests/golden/c2_sampled_rows.json) regenerate from their seed:
x matches the checksum and the rows are the seeded ones plus the points closest to each
interface.  (The oracle's row helper that wrote the values is pinned against the dense
matrix in test_oracle_rows.py.)"""

import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c2_sampled_rows.json")


def test_seed_regenerates_the_sample():
    if not os.path.exists(GOLDEN):
        pytest.skip("c2_sampled_rows.json not generated")
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_c2_sampled_rows as gen
    from oracle import nystrom as onys
    from workloads import config_c2

    with open(GOLDEN) as f:
        d = json.load(f)
    wl = config_c2()
    pts, _, _, _ = onys.elements(wl.bodies)
    x, rows = gen.sample(pts, wl.medium.interfaces)
    assert d["seed"] == gen.SEED and d["n"] == pts.shape[0] == x.size
    assert np.allclose([np.sum(x).real, np.sum(x).imag], d["x_checksum"], rtol=1e-12, atol=1e-9)
    assert list(rows) == d["rows"] and len(d["y"]) == 12
    # the last four rows are the points closest to the interfaces y = 0 and y = -2, one per side
    y = pts[rows[-4:], 1]
    assert y[0] > 0 > y[1] and y[2] > -2 > y[3]
    assert np.all(np.abs(y - np.array([0.0, 0.0, -2.0, -2.0])) < 0.05)
