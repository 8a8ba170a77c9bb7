"""The quadrant form of the cell-to-cell M2M and L2L translations, on the CPU.

The library translates a parent cell and its children as one family (csrc/fmm_kernels.cuh:
fam_up / fam_dn, csrc/mixed.cu: fam_up32 / fam_dn32). The four child offsets (+-w/2, +-w/2)
share one length, so Graf's addition theorem (Sec. 4.1) gives every child the vector of the
quadrant-3 child times a phase. The kernels apply that phase as 4-point transforms with fixed
coefficients. These tests restate those coefficients and the lane-to-quadrant map, and check
them against the per-child sums built directly from Bessel functions.
"""

import numpy as np
import pytest
from scipy.special import jv


def graf(k, dx, dy, hw, sgn):
    """J_m(k rho) e^{i sgn m theta}, m = -hw..hw (index m + hw)."""
    rho, th = np.hypot(dx, dy), np.arctan2(dy, dx)
    m = np.arange(-hw, hw + 1)
    return jv(m, k * rho) * np.exp(1j * sgn * m * th)


def child_offset(q, w):
    """Offset of the child in quadrant q = (ix & 1) | ((iy & 1) << 1) from its parent's centre."""
    return (0.5 * w if q & 1 else -0.5 * w), (0.5 * w if q & 2 else -0.5 * w)


def per_child_m2m(M, k, w, pP, pC):
    """M^P_n = sum_q sum_m M^q_m V^q_{n-m}, V^q_j = J_j(k|d_q|) e^{-i j theta_q}."""
    hw = pP + pC
    out = np.zeros(2 * pP + 1, complex)
    for q, Mq in M.items():
        V = graf(k, *child_offset(q, w), hw, -1)
        for ni in range(2 * pP + 1):
            for mi in range(2 * pC + 1):
                out[ni] += Mq[mi] * V[(ni - pP) - (mi - pC) + hw]
    return out


def per_child_l2l(L, k, w, pP, pC):
    """L^q_n = sum_m L^P_m U^q_{m-n}, U^q_j = J_j(k|d_q|) e^{+i j theta_q}."""
    hw = pP + pC
    res = {}
    for q in range(4):
        U = graf(k, *child_offset(q, w), hw, +1)
        res[q] = np.array([sum(L[mi] * U[(mi - pP) - (ni - pC) + hw] for mi in range(2 * pP + 1))
                           for ni in range(2 * pC + 1)])
    return res


def quad_m2m(M, k, w, pP, pC):
    """The kernels' form: the transforms S^s of the children (om_q = 1, -i, -1, i for the
    quadrants 3, 2, 0, 1), then one Toeplitz sum with the quadrant-3 vector, term (n, m)
    taking S^{(n - m) mod 4}."""
    hw = pP + pC
    z = np.zeros(2 * pC + 1, complex)
    m0, m1, m2, m3 = (M.get(q, z) for q in range(4))
    u, v, x, iy = m3 + m0, m2 + m1, m3 - m0, 1j * (m2 - m1)
    S = [u + v, x - iy, u - v, x + iy]
    B = graf(k, 0.5 * w, 0.5 * w, hw, -1)
    out = np.zeros(2 * pP + 1, complex)
    for ni in range(2 * pP + 1):
        for s in range(4):
            for mi in range((ni - pP + pC - s) & 3, 2 * pC + 1, 4):
                out[ni] += S[s][mi] * B[(ni - pP) - (mi - pC) + hw]
    return out


def quad_l2l(L, k, w, pP, pC):
    """The kernels' form: residue sums T_s (s = (m - n) mod 4) with the quadrant-3 vector, then
    the lane transform, after which lane s holds the child of quadrant 3, 0, 2, 1."""
    hw = pP + pC
    C = graf(k, 0.5 * w, 0.5 * w, hw, +1)
    res = {q: np.zeros(2 * pC + 1, complex) for q in range(4)}
    for ni in range(2 * pC + 1):
        T = [0j, 0j, 0j, 0j]
        for s in range(4):
            for mi in range((ni - pC + pP + s) & 3, 2 * pP + 1, 4):
                T[s] += L[mi] * C[(mi - pP) - (ni - pC) + hw]
        # lane s: b = T_s + T_{s^2} (s < 2) or T_{s^2} - T_s; then with b' of lane s^1
        b = [T[0] + T[2], T[1] + T[3], T[0] - T[2], T[1] - T[3]]
        lane = [b[0] + b[1], b[0] - b[1], b[2] + 1j * b[3], b[2] - 1j * b[3]]
        for s in range(4):
            q = (0x1203 >> (4 * s)) & 15
            res[q][ni] = lane[s]
    return res


CASES = [(4.0, 0.35, 20, 20), (8.0, 0.9, 29, 20), (6.0, 2.1, 57, 37), (12.0, 0.05, 20, 20)]


@pytest.mark.parametrize("k,w,pP,pC", CASES)
def test_quadrant_vectors_are_phases_of_the_base_vector(k, w, pP, pC):
    hw = pP + pC
    j = np.arange(-hw, hw + 1)
    B = graf(k, 0.5 * w, 0.5 * w, hw, -1)
    om = {3: 1 + 0j, 2: -1j, 0: -1 + 0j, 1: 1j}   # M2M; L2L uses the conjugates
    for q in range(4):
        V = graf(k, *child_offset(q, w), hw, -1)
        assert np.allclose(V, B * om[q] ** j, rtol=1e-13, atol=1e-15 * np.abs(B).max())
        U = graf(k, *child_offset(q, w), hw, +1)
        assert np.allclose(U, np.conj(B) * np.conj(om[q]) ** j, rtol=1e-13, atol=1e-15 * np.abs(B).max())


@pytest.mark.parametrize("k,w,pP,pC", CASES)
@pytest.mark.parametrize("children", [(0, 1, 2, 3), (1, 2), (3,), (0, 2, 3)])
def test_m2m_transform_equals_per_child_sum(k, w, pP, pC, children):
    rng = np.random.default_rng(7 + len(children))
    M = {q: rng.standard_normal(2 * pC + 1) + 1j * rng.standard_normal(2 * pC + 1) for q in children}
    ref = per_child_m2m(M, k, w, pP, pC)
    got = quad_m2m(M, k, w, pP, pC)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("k,w,pP,pC", CASES)
def test_l2l_lane_transform_equals_per_child_sum(k, w, pP, pC):
    rng = np.random.default_rng(11)
    L = rng.standard_normal(2 * pP + 1) + 1j * rng.standard_normal(2 * pP + 1)
    ref = per_child_l2l(L, k, w, pP, pC)
    got = quad_l2l(L, k, w, pP, pC)
    for q in range(4):
        assert np.abs(got[q] - ref[q]).max() <= 1e-13 * np.abs(ref[q]).max()


def test_a_wrong_lane_map_is_detected():
    """The check can fail: exchanging the children of lanes 2 and 3 (quadrants 2 and 1) breaks it."""
    k, w, pP, pC = 4.0, 0.35, 20, 20
    rng = np.random.default_rng(3)
    L = rng.standard_normal(2 * pP + 1) + 1j * rng.standard_normal(2 * pP + 1)
    ref = per_child_l2l(L, k, w, pP, pC)
    got = quad_l2l(L, k, w, pP, pC)
    assert np.abs(got[1] - ref[2]).max() > 1e-3 * np.abs(ref[2]).max()
