"""Pins for the oracle's combined-field operator (opt-in second-kind form; the
paper's own system is the single layer).

The field-point gradient of G^r is fixed by the closed-form image solutions of an
equal-k two-layer medium and by finite differences of the (separately pinned)
values in a general three-layer medium; the assembled operator, its jump term
and the field representation by the sound-soft circle series and the layered
manufactured solution, both of which must converge at first order like the
single-layer discretisation.
"""

import json
import os

import numpy as np
import pytest
from scipy.special import hankel1

from oracle import background, combined, core, green, nystrom
from workloads import Medium
from workloads.geometry import circle

from .test_oracle_solve import _circle_series

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dH0i(k, dx, dy):
    """Gradient of (i/4) H_0(k r) with respect to the field point, r = |(dx, dy)|."""
    r = np.hypot(dx, dy)
    d = -0.25j * k * hankel1(1, k * r)
    return d * dx / r, d * dy / r


def test_gradient_equal_k_images():
    # equal k: reflection and transmission are exact images / scaled free waves,
    # so their gradients are gradients of Hankel functions of the image distance
    k, e0, e1 = 3.0, 1.0, 2.5
    m = Medium(interfaces=[0.0], k=[k, k], eta=[e0, e1])
    rng = np.random.default_rng(5)
    n = 40
    x, xs = rng.uniform(-3, 3, n), rng.uniform(-3, 3, n)
    y, ys = rng.uniform(0.05, 2, n), rng.uniform(0.05, 2, n)
    yb, ysb = rng.uniform(-2, -0.05, n), rng.uniform(-2, -0.05, n)
    R = (e0 - e1) / (e0 + e1)
    cases = [
        (x, y, xs, ys, R, y + ys),                        # both above: image below the interface
        (x, yb, xs, ys, 2 * e0 / (e0 + e1), yb - ys),     # field below, source above
        (xs, ys, x, yb, 2 * e1 / (e0 + e1), ys - yb),     # field above, source below
        (x, yb, xs, ysb, -R, yb + ysb),                   # both below
    ]
    for fx, fy, sx, sy, coef, ddy in cases:
        gx, gy = core.gr_grad_block(m, fx, fy, sx, sy)
        gx, gy = np.diag(gx), np.diag(gy)
        ex, ey = dH0i(k, fx - sx, ddy)
        np.testing.assert_allclose(gx, coef * ex, rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(gy, coef * ey, rtol=1e-11, atol=1e-14)


def test_gradient_finite_differences_three_layers():
    m = Medium(interfaces=[0.0, -1.5], k=[3.0, 5.5, 4.0], eta=[1.0, 2.0, 3.0])
    rng = np.random.default_rng(6)
    bands = [(0.1, 2.0), (-1.4, -0.1), (-3.0, -1.6)]
    f, s = [], []
    for lf in range(3):
        for ls in range(3):
            for _ in range(3):
                f.append((rng.uniform(-2, 2), rng.uniform(*bands[lf])))
                s.append((rng.uniform(-2, 2), rng.uniform(*bands[ls])))
    f, s = np.array(f), np.array(s)
    gx, gy = core.gr_grad_block(m, f[:, 0], f[:, 1], s[:, 0], s[:, 1])
    gx, gy = np.diag(gx), np.diag(gy)
    h = 1e-5

    def val(dx, dy):
        return core.gr_pairs(m, f[:, 0] + dx, f[:, 1] + dy, s[:, 0], s[:, 1])

    fdx = (val(h, 0) - val(-h, 0)) / (2 * h)
    fdy = (val(0, h) - val(0, -h)) / (2 * h)
    scale = np.maximum(np.abs(fdx), np.abs(fdy)) + 1e-3
    assert np.max(np.abs(gx - fdx) / scale) < 1e-6
    assert np.max(np.abs(gy - fdy) / scale) < 1e-6
    assert np.min(np.abs(gy)) > 1e-4   # nothing trivially zero


def test_circle_combined_field_first_order():
    # one layer: the combined-field solution's field converges to the series like
    # the single-layer one (a wrong jump sign or a missing 1/2 does not converge)
    k, a, th = 2.0, 0.5, np.deg2rad(30.0)
    m = Medium(interfaces=[], k=[k], eta=[1.0])
    phi = np.linspace(0, 2 * np.pi, 16, endpoint=False)
    r = np.full(16, 2 * a)
    tg = np.stack([r * np.cos(phi), r * np.sin(phi)], 1)
    ex = _circle_series(k, a, -th, r, phi)
    errs, conds = [], []
    for n in [128, 256, 512]:
        pts, w, nrm, _ = nystrom.elements([circle(0, 0, a, n)])
        K = combined.dense_matrix_cf(m, pts, w, nrm)
        b = background.rhs(m, th, pts[:, 0], pts[:, 1])
        Phi = np.linalg.solve(K, b)
        errs.append(np.max(np.abs(combined.field_cf(m, pts, w, nrm, Phi, tg) - ex)))
        conds.append(np.linalg.cond(K))
    assert errs[-1] < 5e-3
    assert 1.6 < errs[1] / errs[2] < 2.6
    # second kind: the condition number stays bounded as the mesh is refined
    assert conds[-1] < 1.2 * conds[0] and conds[-1] < 20


def test_layered_manufactured_solution_combined_field():
    # as the single-layer pin (Sec. 5, Example-1 style) with the combined-field operator
    m = Medium(interfaces=[0.0], k=[2.0, 3.0], eta=[1.0, 2.0])
    src = np.array([0.1, 0.2])
    tg = np.array([[1.5, 0.9], [-1.4, 0.6], [1.2, -1.0], [-0.9, -1.3]])
    ex = green.G(m, tg[:, 0], tg[:, 1], src[0], src[1])
    errs = []
    for n in [64, 128, 256]:
        pts, w, nrm, _ = nystrom.elements([circle(0.0, 0.15, 0.6, n)])
        K = combined.dense_matrix_cf(m, pts, w, nrm)
        lay = green.layer_of(m, pts[:, 1])
        b = m.eta[lay] * green.G(m, pts[:, 0], pts[:, 1], src[0], src[1])
        Phi = np.linalg.solve(K, b)
        errs.append(np.max(np.abs(combined.field_cf(m, pts, w, nrm, Phi, tg) - ex)))
    assert 1.5 < errs[1] / errs[2] < 2.6
    assert errs[-1] < 5e-3


def test_rows_match_dense():
    m = Medium(interfaces=[0.0], k=[2.0, 3.0], eta=[1.0, 2.0])
    pts, w, nrm, _ = nystrom.elements([circle(0.0, 0.15, 0.6, 48)])
    K = combined.dense_matrix_cf(m, pts, w, nrm)
    rows = np.array([0, 7, 30])
    np.testing.assert_allclose(combined.dense_rows_cf(m, pts, w, nrm, rows), K[rows], rtol=0, atol=1e-14)


def test_gradient_transmission_conditions():
    # the analytic field-point gradient obeys the interface conditions of Sec. 3.1:
    # d/dx G and eta dG/dy are continuous across every interface (free part included
    # when the field point's layer holds the source)
    m = Medium(interfaces=[0.0, -0.9, -1.7], k=[3.0, 5.5, 2.0, 4.2], eta=[1.0, 2.5, 1.3, 3.0])
    rng = np.random.default_rng(8)
    bands = [(0.1, 1.5), (-0.8, -0.1), (-1.6, -1.0), (-3.0, -1.8)]

    def grad(x, y, xs, ys):
        gx, gy = core.gr_grad_block(m, [x], [y], [xs], [ys])
        gx, gy = gx[0, 0], gy[0, 0]
        lf, ls = green.layer_of(m, y), green.layer_of(m, ys)
        if lf == ls:
            fx, fy = dH0i(m.k[lf], x - xs, y - ys)
            gx, gy = gx + fx, gy + fy
        return gx, gy

    for ls in range(4):
        xs, ys = rng.uniform(-1, 1), rng.uniform(*bands[ls])
        for j, yi in enumerate(m.interfaces):
            x = rng.uniform(-1, 1)
            ax, ay = grad(x, yi + 1e-12, xs, ys)
            bx, by = grad(x, yi - 1e-12, xs, ys)
            sc = max(abs(ay), abs(ax), 1e-3)
            assert abs(ax - bx) < 1e-9 * sc, (ls, j, ax, bx)
            assert abs(m.eta[j] * ay - m.eta[j + 1] * by) < 1e-9 * max(abs(m.eta[j] * ay), 1e-3), (ls, j)
