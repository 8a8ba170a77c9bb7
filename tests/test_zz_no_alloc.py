"""lfmm_matvec_static: the matvec for callers that cannot allocate device memory.

Real-time threads that must stay out of the allocator (an allocation can block
and synchronise the device), hosts with a fixed memory budget, or frameworks whose
own pool owns the device memory cannot let the library allocate its work buffers
on the first matvec.  lfmm_matvec_static uses one fixed device array instead.
These tests call it through the C ABI: on a freshly built geometry, twice in a
row, each result equal bit for bit to lfmm_matvec on the same input (both run the
same kernels with sums in a fixed order); device memory in use does not change
across a call; a geometry whose work buffers exceed the array is refused before
any device work, with y left untouched.  The file is collected after the other
tests.
"""

import numpy as np
import pytest

from workloads import Medium, config_c1, config_c2, layered_small

pytestmark = pytest.mark.gpu


def _geometry(lf, wl, p, leaf, medium=None):
    med = medium or wl.medium
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    return lf.geometry_build(M, pts, w, nrm, p=p, leaf_size=leaf)


@pytest.mark.parametrize("case", ["fmm_three_layers", "direct_c1"])
def test_static_matvec_matches_matvec(gpu_lib, case):
    import torch

    lf = gpu_lib
    if case == "fmm_three_layers":
        G = _geometry(lf, layered_small(n_bodies=3, nodes=150, seed=7), 20, 16)
        tp = lf.geometry_query(G, "tree_params", np.float64)
        assert tp[4] <= tp[3], "the FMM far field must be exercised"
    else:
        G = _geometry(lf, config_c1(), 20, 64)
    rng = np.random.default_rng(11)
    xs = [torch.from_numpy(rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)).cuda() for _ in range(2)]
    # the allocation-free call comes first on the fresh geometry, twice in a row
    ys = [torch.empty_like(x) for x in xs]
    for x, y in zip(xs, ys):
        lf.matvec_static(G, x, y)
    torch.cuda.synchronize()
    for call, (x, y) in enumerate(zip(xs, ys)):
        y_ref = lf.matvec(G, x)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy(), y_ref.cpu().numpy()), (case, call)
    # and again after lfmm_matvec has allocated the geometry's own buffers
    y2 = torch.empty_like(xs[0])
    lf.matvec_static(G, xs[0], y2)
    torch.cuda.synchronize()
    assert np.array_equal(y2.cpu().numpy(), ys[0].cpu().numpy())


def test_static_matvec_allocates_nothing(gpu_lib):
    import torch

    lf = gpu_lib
    # first call on the device: looks up the array's address and loads the kernels
    Ga = _geometry(lf, layered_small(n_bodies=3, nodes=150, seed=7), 20, 16)
    xa = torch.zeros(Ga.n, dtype=torch.complex128, device="cuda")
    lf.matvec_static(Ga, xa, torch.empty_like(xa))
    Gb = _geometry(lf, layered_small(n_bodies=3, nodes=170, seed=9), 20, 16)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal(Gb.n) + 1j * rng.standard_normal(Gb.n)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    lf.matvec_static(Gb, x, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device memory in use changed by {free0 - free1} bytes"
    assert np.array_equal(y.cpu().numpy(), lf.matvec(Gb, x).cpu().numpy())


def test_static_matvec_refuses_geometry_beyond_the_array(gpu_lib):
    import torch

    lf = gpu_lib
    # one layer, 65,536 points, leaves of at most 8 points at order 40: the multipole and
    # local coefficients alone need far more than the 32 MiB array
    wl = config_c2()
    G = _geometry(lf, wl, 40, 8, medium=Medium(interfaces=[], k=[4.0], eta=[1.0]))
    x = torch.ones(G.n, dtype=torch.complex128, device="cuda")
    y = torch.full((G.n,), 7.0 + 3.0j, dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(lf.LfmmError) as err:
        lf.matvec_static(G, x, y)
    assert err.value.status == lf.LFMM_ERR_INVALID_ARG
    assert "bytes of work memory" in str(err.value)
    torch.cuda.synchronize()
    assert bool(torch.all(y == (7.0 + 3.0j)))
    # the geometry itself is fine for lfmm_matvec
    assert bool(torch.isfinite(torch.view_as_real(lf.matvec(G, x))).all())


def test_static_matvec_checks_vectors_before_the_call(gpu_lib):
    import torch

    lf = gpu_lib
    G = _geometry(lf, config_c1(), 20, 64)
    x = torch.zeros(G.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(TypeError):
        lf.matvec_static(G, x.to(torch.complex64), y)
    with pytest.raises(TypeError):
        lf.matvec_static(G, torch.zeros(2 * G.n, dtype=torch.complex128, device="cuda")[::2], y)
    with pytest.raises(ValueError):
        lf.matvec_static(G, torch.zeros(2 * G.n, dtype=torch.complex128, device="cuda"), y)
