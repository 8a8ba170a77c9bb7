"""Pins for the special functions the oracle relies on (H_0^(1) from scipy)."""

import math

import numpy as np
import pytest
from scipy.special import hankel1, jv, yv

from oracle.green import gf
from oracle.nystrom import EULER_GAMMA

pytestmark = pytest.mark.filterwarnings("ignore")


def _series_j0_y0(z):
    """Ascending series of J_0 and Y_0 (Abramowitz & Stegun 9.1.10, 9.1.13)."""
    z = float(z)
    q = (z / 2.0) ** 2
    j0, term = 0.0, 1.0
    y_sum, harm = 0.0, 0.0
    for kk in range(0, 80):
        if kk > 0:
            term *= -q / (kk * kk)
            harm += 1.0 / kk
        j0 += term
        if kk > 0:
            y_sum += -term * harm
    y0 = (2.0 / math.pi) * (math.log(z / 2.0) + EULER_GAMMA) * j0 + (2.0 / math.pi) * y_sum
    return j0, y0


@pytest.mark.parametrize("z", [1e-3, 0.1, 0.7, 1.9, 3.3, 5.5, 7.9])
def test_h0_against_series(z):
    j0, y0 = _series_j0_y0(z)
    h = hankel1(0, z)
    assert abs(h.real - j0) <= 1e-13 * max(1.0, abs(j0))
    assert abs(h.imag - y0) <= 1e-12 * max(1.0, abs(y0))


def test_wronskian():
    z = np.linspace(0.05, 60.0, 301)
    w = jv(1, z) * yv(0, z) - jv(0, z) * yv(1, z)
    assert np.max(np.abs(w * np.pi * z / 2.0 - 1.0)) < 1e-12


def test_large_argument_asymptotics():
    z = 400.0
    mu = 0.0
    # Hankel asymptotic expansion, three terms (A&S 9.2.7 with P, Q series)
    P = 1.0 - (mu - 1.0) * (mu - 9.0) / (2.0 * (8.0 * z) ** 2)
    Q = (mu - 1.0) / (8.0 * z)
    approx = math.sqrt(2.0 / (math.pi * z)) * (P + 1j * Q) * np.exp(1j * (z - math.pi / 4.0))
    assert abs(hankel1(0, z) - approx) < 1e-9


def test_gf_small_argument_log():
    # (i/4) H_0(kr) ~ i/4 - (1/2pi)(ln(kr/2) + gamma) as r -> 0 (paper, Sec. 3.3)
    k, r = 3.0, 1e-7
    approx = 0.25j - (math.log(k * r / 2.0) + EULER_GAMMA) / (2.0 * math.pi)
    assert abs(gf(k, r) - approx) < 1e-12
