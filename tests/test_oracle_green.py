"""Pins for the oracle's layered Green's function (Sec. 3.1).

Each test fixes the oracle against something other than itself: closed-form
image solutions, invariants (reciprocity, transmission conditions), the
paper's recursions (which the oracle does not use) and the paper's
zero-component count.
"""

import numpy as np
import pytest
from scipy.special import hankel1

from oracle import core, green, paper_forms
from workloads import Medium


def H0i(k, r):
    return 0.25j * hankel1(0, k * r)


def test_single_layer_has_no_reaction():
    m = Medium(interfaces=[], k=[3.0], eta=[1.0])
    g = core.gr_pairs(m, [0.3], [0.1], [-0.4], [0.7])
    assert g[0] == 0


def test_two_layers_equal_k_image_closed_form():
    # equal k: R = (eta0-eta1)/(eta0+eta1) and T are lambda independent, so the
    # reflected field is an exact image source and the transmitted one a scaled
    # free-space wave.
    k, e0, e1 = 3.0, 1.0, 2.5
    m = Medium(interfaces=[0.0], k=[k, k], eta=[e0, e1])
    rng = np.random.default_rng(0)
    n = 60
    x, xs = rng.uniform(-3, 3, n), rng.uniform(-3, 3, n)
    y, ys = rng.uniform(0.05, 2, n), rng.uniform(0.05, 2, n)
    yb = rng.uniform(-2, -0.05, n)
    R = (e0 - e1) / (e0 + e1)
    g = core.gr_pairs(m, x, y, xs, ys)
    np.testing.assert_allclose(g, R * H0i(k, np.hypot(x - xs, y + ys)), rtol=1e-12, atol=1e-14)
    g = core.gr_pairs(m, x, yb, xs, ys)  # field below, source above: T_{01}
    np.testing.assert_allclose(g, 2 * e0 / (e0 + e1) * H0i(k, np.hypot(x - xs, yb - ys)),
                               rtol=1e-12, atol=1e-14)
    g = core.gr_pairs(m, xs, ys, x, yb)  # field above, source below: T_{10}
    np.testing.assert_allclose(g, 2 * e1 / (e0 + e1) * H0i(k, np.hypot(x - xs, yb - ys)),
                               rtol=1e-12, atol=1e-14)
    ysb = rng.uniform(-2, -0.05, n)
    g = core.gr_pairs(m, x, yb, xs, ysb)  # both below: reflection R_{10} off the interface
    np.testing.assert_allclose(g, -R * H0i(k, np.hypot(x - xs, yb + ysb)), rtol=1e-12, atol=1e-14)


def test_three_layers_equal_k_image_series():
    # source and field in the middle slab: multiple reflections between the two
    # interfaces give a geometric series of image sources.
    k = 2.5
    e = [1.0, 3.0, 1.7]
    H = 1.3
    m = Medium(interfaces=[0.0, -H], k=[k, k, k], eta=e)
    Ru = (e[1] - e[0]) / (e[1] + e[0])
    Rd = (e[1] - e[2]) / (e[1] + e[2])
    rng = np.random.default_rng(1)
    n = 25
    x, xs = rng.uniform(-2, 2, n), rng.uniform(-2, 2, n)
    y, ys = rng.uniform(-H + 0.05, -0.05, n), rng.uniform(-H + 0.05, -0.05, n)
    X = x - xs
    hu, hd = y + H, -y  # field: above bottom, below top
    su, sd = -ys, ys + H  # source: to top, to bottom
    ref = np.zeros(n, dtype=np.complex128)
    for j in range(80):
        r = (Ru * Rd) ** j
        ref += Rd * r * H0i(k, np.hypot(X, hu + sd + 2 * j * H))
        ref += Ru * r * H0i(k, np.hypot(X, hd + su + 2 * j * H))
        ref += Ru * Rd * r * H0i(k, np.hypot(X, hu + su + H + 2 * j * H))
        ref += Ru * Rd * r * H0i(k, np.hypot(X, hd + sd + H + 2 * j * H))
    g = core.gr_pairs(m, x, y, xs, ys)
    np.testing.assert_allclose(g, ref, rtol=1e-11, atol=1e-13)


@pytest.fixture(scope="module")
def med3():
    return Medium(interfaces=[0.0, -0.9, -1.7], k=[3.0, 5.5, 2.0, 4.2], eta=[1.0, 2.5, 1.3, 3.0])


def _rand_in_layer(rng, l, n):
    lo = [0.02, -0.88, -1.68, -3.0][l]
    hi = [1.5, -0.02, -0.92, -1.72][l]
    return rng.uniform(lo, hi, n)


def test_reciprocity(med3):
    # eta_l G_{l l'}(r, r') = eta_{l'} G_{l' l}(r', r)   (the operator div(eta grad) + eta k^2
    # is self-adjoint; plain symmetry when l = l')
    rng = np.random.default_rng(2)
    eta = med3.eta
    for lf in range(4):
        for ls in range(4):
            x, xs = rng.uniform(-2, 2, 3), rng.uniform(-2, 2, 3)
            y, ys = _rand_in_layer(rng, lf, 3), _rand_in_layer(rng, ls, 3)
            a = eta[lf] * green.G(med3, x, y, xs, ys)
            b = eta[ls] * green.G(med3, xs, ys, x, y)
            np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)


def test_transmission_conditions(med3):
    # [G] = 0 and [eta dG/dy] = 0 across every interface (Sec. 3.1); one-sided
    # fourth-order differences on each side of the interface.
    rng = np.random.default_rng(3)
    h = 2e-3
    yint = med3.interfaces
    for ls in range(4):
        xs, ys = rng.uniform(-1, 1), _rand_in_layer(rng, ls, 1)[0]
        for j, yi in enumerate(yint):
            x = rng.uniform(-1, 1)
            if abs(yi - ys) < 0.1:
                continue
            above = yi + h * np.arange(0, 5)
            below = yi - h * np.arange(0, 5)
            above[0] += 1e-12
            below[0] -= 1e-12
            ga = green.G(med3, np.full(5, x), above, np.full(5, xs), np.full(5, ys))
            gb = green.G(med3, np.full(5, x), below, np.full(5, xs), np.full(5, ys))
            c = np.array([-25.0, 48.0, -36.0, 16.0, -3.0]) / (12.0 * h)  # one-sided d/dy
            da = c @ ga
            db = -(c @ gb)
            assert abs(ga[0] - gb[0]) < 1e-9 * max(1.0, abs(ga[0]))
            assert abs(med3.eta[j] * da - med3.eta[j + 1] * db) < 2e-6 * max(1.0, abs(da))


def test_helmholtz_equation(med3):
    # (Delta + k_l^2) G = 0 away from the source: 5-point Laplacian, h = 1e-3
    rng = np.random.default_rng(4)
    h = 1e-3
    for lf, ls in [(0, 0), (1, 1), (2, 0), (3, 1), (1, 3)]:
        x, y = rng.uniform(-1, 1), _rand_in_layer(rng, lf, 1)[0]
        y = float(np.clip(y, [0.05, -0.8, -1.6, -3.0][lf], [1.4, -0.1, -1.0, -1.8][lf]))
        xs, ys = x + 0.6, _rand_in_layer(rng, ls, 1)[0]
        X = np.array([x, x + h, x - h, x, x])
        Y = np.array([y, y, y, y + h, y - h])
        g = green.G(med3, X, Y, np.full(5, xs), np.full(5, ys))
        lap = (g[1] + g[2] + g[3] + g[4] - 4 * g[0]) / h ** 2
        k = med3.k[lf]
        assert abs(lap + k * k * g[0]) < 1e-4 * max(1.0, abs(k * k * g[0]))


def test_paper_recursions_match_direct_solve(med3):
    # the paper's R~, T~ recursions and the densities of Cases I-III (with the
    # readings documented in oracle/paper_forms.py) reproduce the direct solve
    rng = np.random.default_rng(5)
    for lf in range(4):
        for ls in range(4):
            for _ in range(4):
                y, ys = _rand_in_layer(rng, lf, 1)[0], _rand_in_layer(rng, ls, 1)[0]
                lam = rng.uniform(0, 9) - 1j * rng.uniform(0, 0.5)
                a = green.gr_spectral(med3, lam, y, ys)[0]
                b = paper_forms.reaction_spectral(med3, lam, lf, ls, y, ys)
                assert abs(a - b) <= 1e-12 * max(abs(a), 1e-12)


def test_paper_density_without_i_is_wrong(med3):
    # reading of the printed 1/(2 k_{l',y}): without the factor i the uniform
    # form disagrees with the direct solve by exactly a factor -i.
    lam = 1.7 - 0.1j
    y, ys = 0.4, 0.8
    a = green.gr_spectral(med3, lam, y, ys)[0]
    b = paper_forms.reaction_spectral(med3, lam, 0, 0, y, ys)
    assert abs(b / 1j - a) > 0.1 * abs(a)


@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_zero_component_count(L):
    # Remark in Sec. 3.1: 4 L^2 non-zero components out of 4 (L+1)^2
    tot = sum(len(paper_forms.nonzero_components(L, l, lp))
              for l in range(L + 1) for lp in range(L + 1))
    assert tot == 4 * L * L


def test_zero_components_vanish(med3):
    # the amplitudes the remark sets to zero are zero in the direct solve too
    lam = np.array([1.3 - 0.05j, 4.0 - 0.2j])
    L = 3
    for lf in range(4):
        for ls in range(4):
            S = core.spectral_amp(med3, lf, ls, lam)
            comps = paper_forms.nonzero_components(L, lf, ls)
            names = ["uu", "ud", "du", "dd"]  # (field, source) order of core.spectral_amp
            for q, nm in enumerate(names):
                if nm not in comps:
                    assert np.all(S[:, q] == 0)
                else:
                    assert np.all(np.abs(S[:, q]) > 0)


def test_sommerfeld_integral_does_not_depend_on_the_contour(med3):
    # Cauchy's theorem: the detour's end T and depth h are choices of the quadrature, not of
    # the quantity.  T x 1.5 and h / 2 move the contour across a region free of poles and
    # branch points (all below T and off the fourth-quadrant detour), so the values must
    # agree to the quadrature tolerance.  A detour that crossed a pole, or a tail that
    # missed part of the integrand, would differ at O(1).
    rng = np.random.default_rng(11)
    xs, ys, xf, yf = [], [], [], []
    for lf in range(4):
        for ls in range(4):
            for _ in range(3):
                yf.append(_rand_in_layer(rng, lf, 1)[0])
                ys.append(_rand_in_layer(rng, ls, 1)[0])
                xf.append(rng.uniform(-2.0, 2.0))
                xs.append(rng.uniform(-2.0, 2.0))
    xf.append(0.4); yf.append(0.3); xs.append(0.4); ys.append(0.6)   # X = 0: real-axis tail rule
    ref = core.gr_pairs(med3, xf, yf, xs, ys)
    scale = np.max(np.abs(ref))
    for t_scale, h_scale in [(1.5, 1.0), (1.0, 0.5), (1.5, 0.5)]:
        g = core.gr_pairs_contour(med3, xf, yf, xs, ys, t_scale, h_scale)
        err = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * scale)
        assert np.max(err) <= 1e-12, (t_scale, h_scale, float(np.max(err)))
    # the default scales are the default contour, bit for bit
    assert np.array_equal(core.gr_pairs_contour(med3, xf, yf, xs, ys, 1.0, 1.0), ref)
