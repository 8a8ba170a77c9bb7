"""Combined-field operator (LFMM_COMBINED_FIELD) on the GPU against the oracle's
dense combined-field matrix, solve and field."""

import numpy as np
import pytest

from oracle import background as obg
from oracle import combined as ocf
from oracle import nystrom as onys
from workloads import config_c2, layered_small, layered_wide

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def small3(gpu_lib):
    lf = gpu_lib
    wl = layered_small(n_bodies=3, nodes=150, seed=7)
    med = wl.medium
    pts, w, nrm, _ = onys.elements(wl.bodies)
    K = ocf.dense_matrix_cf(med, pts, w, nrm)
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    return dict(lf=lf, wl=wl, med=med, pts=pts, w=w, nrm=nrm, K=K, M=M)


def test_all_near_matches_dense_oracle(small3):
    # one leaf: every entry comes from the stored near field, including the
    # Sommerfeld quadrature of the reaction gradients
    lf, s = small3["lf"], small3
    G = lf.geometry_build(s["M"], s["pts"], s["w"], s["nrm"], p=20, leaf_size=1024, combined=True)
    rng = np.random.default_rng(14)
    x = rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)
    err = relerr(lf.matvec(G, x), s["K"] @ x)
    print(f"combined field, all near: {err:.3e}")
    assert err <= 1e-10


@pytest.mark.parametrize("p,tol", [(10, 1e-4), (20, 1e-7)])
def test_fmm_within_truncation_tolerance(small3, p, tol):
    lf, s = small3["lf"], small3
    G = lf.geometry_build(s["M"], s["pts"], s["w"], s["nrm"], p=p, leaf_size=16, combined=True)
    tp = lf.geometry_query(G, "tree_params", np.float64)
    assert tp[4] <= tp[3], "far field must be active"
    rng = np.random.default_rng(15)
    x = rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)
    err = relerr(lf.matvec(G, x), s["K"] @ x)
    print(f"combined field p={p}: {err:.3e}")
    assert err <= tol


def test_wide_band_straddling_cells(gpu_lib):
    lf = gpu_lib
    wl = layered_wide()
    med = wl.medium
    pts, w, nrm, _ = onys.elements(wl.bodies)
    K = ocf.dense_matrix_cf(med, pts, w, nrm)
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, nrm, p=20, leaf_size=8, combined=True)
    rng = np.random.default_rng(16)
    x = rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)
    err = relerr(lf.matvec(G, x), K @ x)
    print(f"combined field, wide band: {err:.3e}")
    assert err <= 1e-8
    # the precision form carries the dipole basis too
    ym = lf.matvec(G, x, mixed=True)
    assert relerr(ym, lf.matvec(G, x)) <= 2e-6


def test_solve_and_field_match_oracle(small3):
    lf, s = small3["lf"], small3
    med, pts, w, nrm, K = s["med"], s["pts"], s["w"], s["nrm"], s["K"]
    G = lf.geometry_build(s["M"], pts, w, nrm, p=20, leaf_size=16, combined=True)
    Gs = lf.geometry_build(s["M"], pts, w, p=20, leaf_size=16)
    b = obg.rhs(med, np.deg2rad(45.0), pts[:, 0], pts[:, 1])
    x, info = lf.gmres_solve(G, b, tol=1e-8)
    xs, infos = lf.gmres_solve(Gs, b, tol=1e-8)
    ref = np.linalg.solve(K, b)
    print("combined field", info, "single layer", infos)
    assert info["converged"] and info["true_rel_residual"] <= 1e-8
    assert relerr(x, ref) <= 1e-6
    # second kind: fewer iterations than the first-kind single layer
    assert info["iterations"] < infos["iterations"]
    tg = np.array([[0.3, 2.5], [-4.0, 1.0], [2.0, -3.5], [5.5, -1.2]])
    u = lf.eval_field(G, x, tg)
    assert relerr(u, ocf.field_cf(med, pts, w, nrm, x, tg)) <= 1e-9
    # both formulations represent the same scattered field (to discretisation error)
    us = lf.eval_field(Gs, xs, tg)
    print("field: combined vs single layer", relerr(u, us))
    assert relerr(u, us) <= 1e-2
    # mixed precision with refinement reaches the same residual
    xm, im = lf.gmres_solve(G, b, tol=1e-8, precision=1)
    assert im["converged"] and im["true_rel_residual"] <= 1e-8
    assert relerr(xm, x) <= 1e-6


def test_c2_full_size_sampled_rows(gpu_lib):
    lf = gpu_lib
    wl = config_c2()
    med = wl.medium
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size, combined=True)
    rng = np.random.default_rng(17)
    x = rng.standard_normal(G.n) + 1j * rng.standard_normal(G.n)
    y = lf.matvec(G, x)
    assert np.array_equal(lf.matvec(G, x), y)
    rows = rng.integers(0, G.n, 2)
    ref = ocf.dense_rows_cf(med, pts, w, nrm, rows) @ x
    err = np.max(np.abs(y[rows] - ref) / np.abs(ref))
    print(f"C2 combined field sampled rows: max rel err {err:.3e}")
    assert err <= 1e-7
