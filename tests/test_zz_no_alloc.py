"""lfmm_matvec_static: the matvec for callers that cannot allocate device memory.

Real-time threads that must stay out of the allocator (an allocation can block
and synchronise the device), hosts with a fixed memory budget, or frameworks whose
own pool owns the device memory cannot let the library allocate its work buffers
on the first matvec.  lfmm_matvec_static uses one
fixed device array instead; this test calls it through the C ABI twice in a
row and checks each result against lfmm_matvec on the same input.  It is kept
in a file of its own, collected after the other tests.
"""

import numpy as np
import pytest

from workloads import config_c1, layered_small

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["fmm_three_layers", "direct_c1"])
def test_static_matvec_matches_matvec(gpu_lib, case):
    import torch

    lf = gpu_lib
    wl = layered_small(n_bodies=3, nodes=150, seed=7) if case == "fmm_three_layers" else config_c1()
    leaf = 16 if case == "fmm_three_layers" else 64
    med = wl.medium
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    G = lf.geometry_build(M, pts, w, nrm, p=20, leaf_size=leaf)
    if case == "fmm_three_layers":
        tp = lf.geometry_query(G, "tree_params", np.float64)
        assert tp[4] <= tp[3], "the FMM far field must be exercised"
    rng = np.random.default_rng(11)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)).cuda()
        y_ref = lf.matvec(G, x)
        y = torch.empty_like(x)
        lf.matvec_static(G, x, y)
        torch.cuda.synchronize()
        assert _relerr(y.cpu().numpy(), y_ref.cpu().numpy()) <= 1e-12, (case, call)
