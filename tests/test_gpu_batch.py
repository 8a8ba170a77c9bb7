"""Several geometries' operators in shared launches (lfmm_matvec_batch) against each
geometry's own lfmm_matvec: uneven sizes, depths and layer counts, all-near and far-field
geometries, different column counts, complex128 and complex64 vectors.  The batched launches
run the same kernel bodies with the same summation order, so the results are equal bit for
bit; the per-geometry products are themselves held to the oracle by the parity tests."""

import numpy as np
import pytest

from workloads import Medium, config_c1, layered_small, layered_wide

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def geos(gpu_lib):
    lf = gpu_lib
    out = []
    for wl, leaf in [(layered_small(n_bodies=3, nodes=150, seed=7), 16),     # three layers, far field
                     (config_c1(), 64),                                       # two layers, all near
                     (layered_wide(), 8),                                     # wide band, straddling cells
                     (layered_small(n_bodies=4, nodes=120, seed=9, n_layers=4), 12),
                     (layered_small(n_bodies=2, nodes=200, seed=3, n_layers=3), 1024)]:   # all near
        med = wl.medium
        M = lf.medium_create(med.interfaces, med.k, med.eta)
        pts, w, nrm = lf.polygon_elements(wl.bodies)
        out.append(lf.geometry_build(M, pts, w, nrm, p=20, leaf_size=leaf))
    one = Medium(interfaces=[], k=[5.0], eta=[1.0])
    wl = layered_small(n_bodies=3, nodes=100, seed=5)
    M = lf.medium_create(one.interfaces, one.k, one.eta)
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    out.append(lf.geometry_build(M, pts, w, nrm, p=20, leaf_size=16))   # one layer
    return out


def _vectors(G, nrhs, seed, dtype):
    import torch

    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nrhs, G.n)) + 1j * rng.standard_normal((nrhs, G.n))
    t = torch.from_numpy(a).to(dtype).cuda()
    return t[0].contiguous() if nrhs == 1 else t


@pytest.mark.parametrize("single", [False, True])
def test_batch_equals_per_geometry_products(gpu_lib, geos, single):
    import torch

    lf = gpu_lib
    dtype = torch.complex64 if single else torch.complex128
    nrhs = [1, 3, 2, 1, 2, 4]
    xs = [_vectors(G, r, 40 + i, dtype) for i, (G, r) in enumerate(zip(geos, nrhs))]
    ys = lf.matvec_batch(geos, xs)
    torch.cuda.synchronize()
    for G, x, y in zip(geos, xs, ys):
        ref = lf.matvec(G, x)
        torch.cuda.synchronize()
        assert torch.equal(y, ref)
    # the batch in another order and a subset give the same bits
    ys2 = lf.matvec_batch(geos[::-2], xs[::-2])
    torch.cuda.synchronize()
    for y2, y in zip(ys2, ys[::-2]):
        assert torch.equal(y2, y)


def test_batch_rejects_a_repeated_geometry(gpu_lib, geos):
    import torch

    lf = gpu_lib
    x = torch.zeros(geos[0].n, dtype=torch.complex128, device="cuda")
    with pytest.raises(lf.LfmmError) as err:
        lf.matvec_batch([geos[0], geos[0]], [x, x.clone()])
    assert err.value.status == lf.LFMM_ERR_INVALID_ARG
