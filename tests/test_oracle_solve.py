"""Pins for the oracle's discretisation, right-hand side and solvers (Secs. 2.2, 3.3, 4.2, 5)."""

import json
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import hankel1, jv, j0, y0

from oracle import background, gmres, green, nystrom, paper_forms, tree
from workloads import Medium, circle, config_c1, layered_small

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_self_term_against_quadrature():
    # I^s drops only the regular part I^r = O(k^2 h^3 ln h) of the exact element
    # integral of (i/4) H_0 (Sec. 3.3); check the size and the h^3 scaling.
    k = 3.0
    errs = []
    for h in [0.08, 0.04, 0.02]:
        re = 2 * quad(lambda s: -0.25 * y0(k * s), 0, h / 2, limit=200, epsabs=1e-15)[0]
        im = 2 * quad(lambda s: 0.25 * j0(k * s), 0, h / 2, limit=200, epsabs=1e-15)[0]
        errs.append(abs(nystrom.self_term(k, h) - (re + 1j * im)))
    assert errs[0] < 5e-4
    assert 5.0 < errs[0] / errs[1] < 12.0 and 5.0 < errs[1] / errs[2] < 12.0


def test_two_layer_fresnel_background():
    # a single interface: the background field is the Fresnel reflection/transmission
    k0, k1, e0, e1 = 2.0, 3.5, 1.0, 2.2
    m = Medium(interfaces=[0.0], k=[k0, k1], eta=[e0, e1])
    th = np.deg2rad(35.0)
    kx = k0 * np.cos(th)
    ky0, ky1 = k0 * np.sin(th), np.sqrt(k1 ** 2 - kx ** 2)
    R = (e0 * ky0 - e1 * ky1) / (e0 * ky0 + e1 * ky1)
    T = 2 * e0 * ky0 / (e0 * ky0 + e1 * ky1)
    x = np.array([0.3, -1.1, 0.7])
    ya, yb = np.array([0.4, 1.3, 0.05]), np.array([-0.4, -1.3, -0.05])
    np.testing.assert_allclose(background.background(m, th, x, ya),
                               R * np.exp(1j * (kx * x + ky0 * ya)), rtol=1e-13)
    np.testing.assert_allclose(background.background(m, th, x, yb),
                               T * np.exp(1j * (kx * x - ky1 * yb)), rtol=1e-13)


def test_background_interface_conditions_and_paper_form():
    m = Medium(interfaces=[0.0, -0.8, -1.9], k=[3.0, 5.0, 2.5, 4.0], eta=[1.0, 2.0, 3.5, 1.5])
    th = np.deg2rad(60.0)
    h = 1e-4
    x = 0.37
    for j, yi in enumerate(m.interfaces):
        ya = np.array([yi + 1e-12, yi + h, yi + 2 * h])
        yb = np.array([yi - 1e-12, yi - h, yi - 2 * h])
        ua = background.background(m, th, x, ya) + background.incident(m, th, x, ya)
        ub = background.background(m, th, x, yb) + background.incident(m, th, x, yb)
        assert abs(ua[0] - ub[0]) < 1e-10
        da = (-3 * ua[0] + 4 * ua[1] - ua[2]) / (2 * h)
        db = -(-3 * ub[0] + 4 * ub[1] - ub[2]) / (2 * h)
        assert abs(m.eta[j] * da - m.eta[j + 1] * db) < 1e-5 * max(1, abs(da))
    # the paper's closed form A_l, B_l (absolute coordinates) agrees with the transfer solve
    kx, kyv, A, B, _ = background.background_coefficients(m, th)
    _, _, A2, B2 = paper_forms.background_paper(m, th)
    yint = m.interfaces
    for l in range(4):
        if l <= 2:
            assert abs(A[l] * np.exp(-1j * kyv[l] * yint[l]) - A2[l]) < 1e-13
        if l >= 1:
            assert abs(B[l] * np.exp(1j * kyv[l] * yint[l - 1]) - B2[l]) < 1e-13


def _circle_series(k, a, th_dir, r, phi):
    n = np.arange(-60, 61)
    c = -(1j ** n) * jv(n, k * a) / hankel1(n, k * a)
    return np.sum(c[None, :] * hankel1(n[None, :], k * r[:, None])
                  * np.exp(1j * n[None, :] * (phi[:, None] - th_dir)), axis=1)


def test_circle_series_first_order():
    # one layer (no reaction): sound-soft circle against its Bessel/Hankel series;
    # the lowest-order Nystrom error decays at first order (Sec. 5).
    k, a, th = 2.0, 0.5, np.deg2rad(30.0)
    m = Medium(interfaces=[], k=[k], eta=[1.0])
    phi = np.linspace(0, 2 * np.pi, 16, endpoint=False)
    r = np.full(16, 2 * a)
    tg = np.stack([r * np.cos(phi), r * np.sin(phi)], 1)
    ex = _circle_series(k, a, -th, r, phi)  # u_inc = exp(i k (x cos th - y sin th))
    errs = []
    for n in [128, 256, 512]:
        pts, w, _, _ = nystrom.elements([circle(0, 0, a, n)])
        K = nystrom.dense_matrix(m, pts, w)
        Phi = np.linalg.solve(K, background.rhs(m, th, pts[:, 0], pts[:, 1]))
        errs.append(np.max(np.abs(nystrom.field(m, pts, w, Phi, tg) - ex)))
    assert errs[-1] < 5e-4
    assert errs[1] / errs[2] > 1.6


def test_layered_manufactured_solution_first_order():
    # Example-1 style manufactured solution (Sec. 5): boundary data g = G(c, r_src)
    # with the source inside a scatterer that crosses an interface; the error of
    # u^s against G(r, r_src) outside decays at first order.
    m = Medium(interfaces=[0.0], k=[2.0, 3.0], eta=[1.0, 2.0])
    src = np.array([0.1, 0.2])
    tg = np.array([[1.5, 0.9], [-1.4, 0.6], [1.2, -1.0], [-0.9, -1.3]])
    ex = green.G(m, tg[:, 0], tg[:, 1], src[0], src[1])
    errs = []
    with open(os.path.join(GOLDEN, "paper_example1_table51.json")) as f:
        paper = json.load(f)
    for n in [64, 128, 256]:
        pts, w, _, _ = nystrom.elements([circle(0.0, 0.15, 0.6, n)])
        K = nystrom.dense_matrix(m, pts, w)
        lay = green.layer_of(m, pts[:, 1])
        b = m.eta[lay] * green.G(m, pts[:, 0], pts[:, 1], src[0], src[1])
        Phi = np.linalg.solve(K, b)
        errs.append(np.max(np.abs(nystrom.field(m, pts, w, Phi, tg) - ex)))
    # the paper's L_inf column halves per doubling of N (Table 5.1)
    ratios = np.array(paper["linf"][:-1]) / np.array(paper["linf"][1:])
    assert np.all((ratios > 1.9) & (ratios < 2.1))
    assert 1.5 < errs[1] / errs[2] < 2.6
    assert errs[-1] < 5e-3


def test_gmres_matches_lu_c1():
    wl = config_c1()
    pts, w, _, _ = nystrom.elements(wl.bodies)
    K = nystrom.dense_matrix(wl.medium, pts, w)
    b = background.rhs(wl.medium, np.deg2rad(45.0), pts[:, 0], pts[:, 1])
    x_lu = np.linalg.solve(K, b)
    x, it, hist, conv = gmres.gmres(lambda v: K @ v, b, tol=1e-10)
    assert conv and it < 100
    assert np.linalg.norm(K @ x - b) / np.linalg.norm(b) <= 1.0001e-10
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-8


def test_dd_preconditioner_reduces_iterations():
    wl = layered_small(n_bodies=3, nodes=160, seed=3)
    pts, w, _, _ = nystrom.elements(wl.bodies)
    m = wl.medium
    K = nystrom.dense_matrix(m, pts, w)
    b = background.rhs(m, np.deg2rad(45.0), pts[:, 0], pts[:, 1])
    T = tree.Tree(pts, m.interfaces, m.k, p=20, leaf_size=16)
    lay = green.layer_of(m, pts[:, 1])
    isd = nystrom.self_term(m.k[lay], w)
    P = tree.dd_preconditioner_dense(T, pts, w, m.k, isd)
    x0, it0, _, c0 = gmres.gmres(lambda v: K @ v, b, tol=1e-8)
    x1, it1, _, c1 = gmres.gmres(lambda v: K @ v, b, tol=1e-8, M=lambda v: P @ v)
    assert c0 and c1
    assert it1 < it0
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-6
    # each leaf's rows reproduce the matching rows of the local inverse
    B = T.boxes_at(T.D)[0]
    J = np.concatenate([T.perm[T.box_begin[S]:T.box_end[S]] for S in T.U_free[B]])
    own = T.perm[T.box_begin[B]:T.box_end[B]]
    PB = nystrom.free_block(m.k[T.box_layer[B]], pts[J], pts[J], w[J], exclude_self=True)
    PB[np.arange(J.size), np.arange(J.size)] = isd[J]
    v = np.random.default_rng(0).standard_normal(J.size) + 0j
    full = np.zeros(pts.shape[0], dtype=np.complex128)
    full[J] = v
    z = np.linalg.solve(PB, v)
    pos = {int(j): a for a, j in enumerate(J)}
    np.testing.assert_allclose((P @ full)[own], z[[pos[int(i)] for i in own]], rtol=1e-10)
