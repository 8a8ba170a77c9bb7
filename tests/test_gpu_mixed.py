"""Precision form (FP32 multipole-to-local translations on scaled expansions) and the
mixed-precision GMRES with iterative refinement, against the FP64 path and the oracle."""

import math

import numpy as np
import pytest

from oracle import nystrom as onys
from workloads import config_c2, layered_wide

pytestmark = pytest.mark.gpu

# bound on ||(A_mixed - A) x|| / ||A x||: FP32 rounding (2^-24 ~ 6e-8) of sums of a
# few thousand terms through the far field, which carries a fraction of the operator
OP_TOL = 2e-6


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def wide(gpu_lib):
    lf = gpu_lib
    wl = layered_wide()
    med = wl.medium
    pts, w, _, _ = onys.elements(wl.bodies)
    K = onys.dense_matrix(med, pts, w)
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, p=20, leaf_size=8)
    return dict(lf=lf, wl=wl, med=med, pts=pts, w=w, K=K, M=M, G=G)


@pytest.fixture(scope="module")
def c2(gpu_lib):
    lf = gpu_lib
    wl = config_c2()
    med = wl.medium
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size)
    return dict(lf=lf, wl=wl, med=med, pts=pts, w=w, M=M, G=G)


def test_mixed_matvec_wide_band_against_fp64_and_oracle(wide):
    lf, G, K = wide["lf"], wide["G"], wide["K"]
    rng = np.random.default_rng(21)
    x = rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)
    y64 = lf.matvec(G, x)
    y32 = lf.matvec(G, x, mixed=True)
    d64, d32 = relerr(y32, y64), relerr(y32, K @ x)
    print(f"wide: mixed vs FP64 {d64:.3e}, mixed vs oracle {d32:.3e}")
    assert d64 <= OP_TOL
    assert d32 <= OP_TOL + 1e-8
    # the FP64 path is untouched by the precision form having been built
    assert np.array_equal(lf.matvec(G, x), y64)


def test_mixed_matvec_c2_against_fp64(c2):
    lf, G = c2["lf"], c2["G"]
    rng = np.random.default_rng(22)
    X = np.asfortranarray(rng.standard_normal((G.n, 2)) + 1j * rng.standard_normal((G.n, 2)))
    y64 = lf.matvec(G, X)
    y32 = lf.matvec(G, X, mixed=True)
    for c in range(2):
        d = relerr(y32[:, c], y64[:, c])
        print(f"C2 column {c}: mixed vs FP64 {d:.3e}")
        assert d <= OP_TOL
    # reproducible
    assert np.array_equal(lf.matvec(G, X, mixed=True), y32)


def test_mixed_gmres_refinement_reaches_fp64_residual_wide(wide):
    lf, G, K = wide["lf"], wide["G"], wide["K"]
    wl = wide["wl"]
    b = lf.rhs_plane_wave(G, [math.radians(float(wl.angles_deg[0]))])
    x1, i1 = lf.gmres_solve(G, b, tol=1e-8, precision=1)
    ref = np.linalg.solve(K, b)
    print("mixed GMRES:", i1)
    assert i1["converged"] and i1["refinements"] >= 1 and i1["fp64_matvecs"] < i1["iterations"]
    assert i1["true_rel_residual"] <= 1e-8
    assert 0.0 < i1["op_rel_diff"] <= OP_TOL
    # residual of the dense oracle matrix
    assert relerr(K @ x1, b) <= 2e-8
    assert relerr(x1, ref) <= 1e-5


def test_mixed_gmres_refinement_c2(c2):
    lf, G, wl = c2["lf"], c2["G"], c2["wl"]
    b = lf.rhs_plane_wave(G, [math.radians(float(wl.angles_deg[0]))])
    x0, i0 = lf.gmres_solve(G, b, tol=1e-8, precision=0)
    x1, i1 = lf.gmres_solve(G, b, tol=1e-8, precision=1)
    print("C2 FP64:", i0)
    print("C2 mixed:", i1)
    assert i0["converged"] and i1["converged"]
    assert i1["true_rel_residual"] <= 1e-8
    assert relerr(x1, x0) <= 1e-5


@pytest.mark.parametrize("ncols", [32, 70])
def test_block_m2l_on_tensor_cores_c2(c2, ncols):
    # 16 or more columns: the FP32 levels' M2L runs on tcgen05 (3xTF32); 70 columns
    # take two launches (64 + 6, the second padded to 16)
    lf, G = c2["lf"], c2["G"]
    rng = np.random.default_rng(24)
    X = np.asfortranarray(rng.standard_normal((G.n, ncols)) + 1j * rng.standard_normal((G.n, ncols)))
    y64 = lf.matvec(G, X)
    ytc = lf.matvec(G, X, mixed=True)
    ysimt = lf.matvec(G, X, mixed=True, simt_m2l=True)
    d64 = max(relerr(ytc[:, c], y64[:, c]) for c in range(ncols))
    dsimt = max(relerr(ytc[:, c], ysimt[:, c]) for c in range(ncols))
    print(f"C2 {ncols} columns: tensor-core mixed vs FP64 {d64:.3e}, vs SIMT mixed {dsimt:.3e}")
    assert d64 <= OP_TOL
    assert dsimt <= 5e-7
    assert np.array_equal(lf.matvec(G, X, mixed=True), ytc)


def test_block_m2l_on_tensor_cores_wide_band(wide):
    # straddling cells (reaction centres), mirrored tables and both departure/arrival flips
    lf, G, K = wide["lf"], wide["G"], wide["K"]
    rng = np.random.default_rng(25)
    X = np.asfortranarray(rng.standard_normal((G.n, 20)) + 1j * rng.standard_normal((G.n, 20)))
    ytc = lf.matvec(G, X, mixed=True)
    ysimt = lf.matvec(G, X, mixed=True, simt_m2l=True)
    ref = K @ X
    for c in range(20):
        assert relerr(ytc[:, c], ref[:, c]) <= OP_TOL + 1e-8
        assert relerr(ytc[:, c], ysimt[:, c]) <= 5e-7


def test_kernel_shared_memory_limits_only_grow_across_geometries(c2):
    # The dynamic shared-memory limit of a kernel is process-wide: building and running a
    # geometry with smaller expansions (smaller P2M/L2P/tensor-core tiles) between two runs of
    # one with larger expansions must leave the larger geometry launchable, with unchanged results.
    lf, G, med, pts, w = c2["lf"], c2["G"], c2["med"], c2["pts"], c2["w"]
    rng = np.random.default_rng(26)
    X = np.asfortranarray(rng.standard_normal((G.n, 16)) + 1j * rng.standard_normal((G.n, 16)))
    y_big = lf.matvec(G, X, mixed=True)
    y_big64 = lf.matvec(G, X)
    small = lf.geometry_build(c2["M"], pts, w, p=12, leaf_size=32)
    y_small = lf.matvec(small, X, mixed=True)
    assert max(relerr(y_small[:, c], y_big64[:, c]) for c in range(16)) <= 1e-2
    assert np.array_equal(lf.matvec(G, X, mixed=True), y_big)
    assert np.array_equal(lf.matvec(G, X), y_big64)


def test_precision_form_near_field_split(gpu_lib):
    # Every pair near (leaf size above N).  In three layers the single block holds
    # reaction (Sommerfeld) entries, so the precision form keeps it in FP64 and equals
    # the FP64 operator to rounding (the two forms split the columns over warps differently).  In one layer the block holds only free-space
    # entries: its off-diagonal entries go to complex64 (FP32 products), the self terms
    # I^s stay FP64, and the difference from the FP64 operator is FP32 rounding.
    from workloads import Medium, layered_small

    lf = gpu_lib
    wl = layered_small(n_bodies=3, nodes=150, seed=7)
    pts, w, _, _ = onys.elements(wl.bodies)
    rng = np.random.default_rng(31)
    x = rng.standard_normal(pts.shape[0]) + 1j * rng.standard_normal(pts.shape[0])
    med = wl.medium
    G3 = lf.geometry_build(lf.medium_create(med.interfaces, med.k, med.eta), pts, w, p=20, leaf_size=1024)
    assert relerr(lf.matvec(G3, x, mixed=True), lf.matvec(G3, x)) <= 1e-14
    one = Medium(interfaces=[], k=[4.0], eta=[1.0])
    K1 = onys.dense_matrix(one, pts, w)
    G1 = lf.geometry_build(lf.medium_create(one.interfaces, one.k, one.eta), pts, w, p=20, leaf_size=1024)
    y64, y32 = lf.matvec(G1, x), lf.matvec(G1, x, mixed=True)
    d, d_or = relerr(y32, y64), relerr(y32, K1 @ x)
    print(f"one layer, all near: precision form vs FP64 {d:.3e}, vs oracle {d_or:.3e}")
    assert 1e-12 < d <= 3e-7 and d_or <= 3e-7
    # the self terms are applied in FP64: on a vector with one non-zero entry the
    # diagonal entry of the product carries no FP32 rounding
    e = np.zeros(pts.shape[0], dtype=np.complex128)
    e[17] = 1.0
    d17 = lf.matvec(G1, e)[17]
    assert lf.matvec(G1, e, mixed=True)[17] == d17
    assert abs(d17 - K1[17, 17]) <= 1e-12 * abs(K1[17, 17])
