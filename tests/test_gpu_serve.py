"""Serving loop (lfmm_server_*): requests of different layer stacks and sizes, run
alone and concurrently; each result must be the same alone and in the mix."""

import math

import numpy as np
import pytest

from workloads import Medium, config_c1, layered_small, layered_wide
from workloads.geometry import random_bodies

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for wl in (config_c1(), layered_small(), layered_wide()):
        out.append((wl.medium, wl.bodies, float(wl.angles_deg[0])))
    # two more in the style of the serving workload (random 2-4 layer stacks, k in [2, 12]),
    # small enough for a quick test
    rng = np.random.default_rng(31)
    for nlay, nb in ((4, 6), (2, 3)):
        interfaces = -2.0 * np.arange(nlay - 1)
        med = Medium(interfaces=interfaces, k=rng.uniform(2.0, 12.0, size=nlay),
                     eta=np.arange(1, nlay + 1, dtype=float))
        bodies = random_bodies(rng, nb, ((-6.0, 6.0), (-5.0, 2.0)), interfaces, 512)
        out.append((med, bodies, float(rng.uniform(5.0, 175.0))))
    return out


def _submit(lf, srv, req, precision):
    med, bodies, ang = req
    pts, w, _ = lf.polygon_elements(bodies)
    return srv.submit(med.interfaces, med.k, med.eta, pts, w, math.radians(ang), tol=1e-8,
                      precision=precision, max_iter=600)


def test_results_alone_equal_results_in_the_mix(gpu_lib):
    lf = gpu_lib
    reqs = _requests()
    precs = [0, 1, 0, 1, 0]
    alone = []
    s1 = lf.Server(slots=1, hbm_budget=64 << 30)
    for r, pr in zip(reqs, precs):
        x, info, t = s1.wait(_submit(lf, s1, r, pr))
        assert info["converged"] and info["true_rel_residual"] <= 1e-8
        alone.append(x)
    assert s1.stats()["peak_running"] == 1
    s1.close()
    srv = lf.Server(slots=3, hbm_budget=64 << 30)
    tickets = [_submit(lf, srv, r, pr) for r, pr in zip(reqs, precs)]
    res = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    print("peak running", st["peak_running"], "latencies", [round(r[2]["latency_seconds"], 3) for r in res])
    assert st["peak_running"] >= 2
    for (x, info, t), xa in zip(res, alone):
        assert info["converged"] and info["true_rel_residual"] <= 1e-8
        assert np.array_equal(x, xa)
        assert t["latency_seconds"] >= t["service_seconds"] > 0.0


def test_server_matches_direct_solve_and_admits_by_footprint(gpu_lib):
    lf = gpu_lib
    wl = layered_small()
    med = wl.medium
    pts, w, _ = lf.polygon_elements(wl.bodies)
    ang = math.radians(float(wl.angles_deg[0]))
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, p=20, leaf_size=64)
    b = lf.rhs_plane_wave(G, [ang])
    xd, _ = lf.gmres_solve(G, b, tol=1e-8, max_iter=600)
    # a budget that holds one request at a time: three slots, but one runs at once
    srv = lf.Server(slots=3, hbm_budget=1)
    with pytest.raises(lf.LfmmError):   # the footprint alone exceeds the budget
        srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, max_iter=600)
    srv.close()
    one = 16 * pts.shape[0] * 601 + 16 * pts.shape[0] * (240 + 24) + 4 * 41 * pts.shape[0] + (300 << 20)
    srv = lf.Server(slots=3, hbm_budget=one)
    ts = [srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, max_iter=600) for _ in range(3)]
    xs = [srv.wait(t)[0] for t in ts]
    assert srv.stats()["peak_running"] == 1
    srv.close()
    for x in xs:
        assert np.array_equal(x, xd)


def test_combined_field_request_matches_direct_solve(gpu_lib):
    lf = gpu_lib
    wl = layered_small()
    med = wl.medium
    pts, w, nrm = lf.polygon_elements(wl.bodies)
    ang = math.radians(float(wl.angles_deg[0]))
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, nrm, p=20, leaf_size=64, combined=True)
    b = lf.rhs_plane_wave(G, [ang])
    xd, infod = lf.gmres_solve(G, b, tol=1e-8, max_iter=600)
    srv = lf.Server(slots=2, hbm_budget=64 << 30)
    with pytest.raises(lf.LfmmError):   # the combined field needs the normals
        srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, combined=True)
    t1 = srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, max_iter=600, normals=nrm, combined=True)
    t2 = srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, max_iter=600)
    x1, i1, _ = srv.wait(t1)
    x2, i2, _ = srv.wait(t2)
    srv.close()
    assert np.array_equal(x1, xd) and i1["iterations"] == infod["iterations"]
    assert i1["converged"] and i2["converged"] and i1["iterations"] < i2["iterations"]
