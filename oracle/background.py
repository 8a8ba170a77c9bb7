"""Plane incidence and background field (Sec. 2.2, eqs. incidentwave, homogeneousscattering).

Test infrastructure only: used by tests/, the smoke check and bench.py's CPU
baseline; the library never imports or calls it.

The incident wave lives in the top layer:
    u_inc = exp(i (k0x x - k0y y)),  k0x = k0 cos(theta), k0y = k0 sin(theta) > 0,
with theta in (0, pi) measured from the +x axis (reading of the incidence
angle; theta = 135 deg gives Example 2's direction, 90 deg Example 3's).

The background field u^b is computed here by a direct transfer solve, not by
the paper's closed form with R~ and T~ (that closed form is implemented in
paper_forms.py and pinned against this solve).  In layer m

    u^b = A_m e^{i(kx x + k_{m,y} (y - y_m))} + B_m e^{i(kx x - k_{m,y} (y - y_{m-1}))}

with y_m the interface below layer m (up-going wave referenced there) and
y_{m-1} the interface above (down-going wave referenced there); A_L = 0 and
B_0 = 0, and u^b + u_inc satisfies [u] = 0, [eta du/dy] = 0 on every interface.
"""

from __future__ import annotations

import numpy as np

from .green import layer_of


def _ky(k, kx):
    s = np.sqrt(np.asarray(k, dtype=np.complex128) ** 2 - kx ** 2)
    return np.where(s.imag < 0, -s, s)


def background_coefficients(medium, theta: float):
    """Return (kx, kyv, A, B, c_inc): amplitudes of the background field."""
    yint = np.asarray(medium.interfaces, dtype=np.float64).reshape(-1)
    k = np.asarray(medium.k, dtype=np.float64)
    eta = np.asarray(medium.eta, dtype=np.float64)
    L = yint.size
    kx = k[0] * np.cos(theta)
    kyv = _ky(k, kx)
    A = np.zeros(L + 1, dtype=np.complex128)
    B = np.zeros(L + 1, dtype=np.complex128)
    if L == 0:
        return kx, kyv, A, B, 1.0 + 0j
    # incident wave as a down-going wave referenced at the first interface
    c_inc = np.exp(-1j * kyv[0] * yint[0])
    e = np.zeros(L + 1, dtype=np.complex128)
    for m in range(1, L):
        e[m] = np.exp(1j * kyv[m] * (yint[m - 1] - yint[m]))
    n = 2 * L
    M = np.zeros((n, n), dtype=np.complex128)
    rhs = np.zeros(n, dtype=np.complex128)

    def ia(m):
        return m

    def ib(m):
        return L + m - 1

    for j in range(L):
        up, lo = j, j + 1
        rc, rf = 2 * j, 2 * j + 1
        M[rc, ia(up)] += 1.0
        M[rf, ia(up)] += eta[up] * 1j * kyv[up]
        if up >= 1:
            M[rc, ib(up)] += e[up]
            M[rf, ib(up)] += -eta[up] * 1j * kyv[up] * e[up]
        if lo <= L - 1:
            M[rc, ia(lo)] -= e[lo]
            M[rf, ia(lo)] -= eta[lo] * 1j * kyv[lo] * e[lo]
        M[rc, ib(lo)] -= 1.0
        M[rf, ib(lo)] -= -eta[lo] * 1j * kyv[lo]
        if j == 0:  # incident wave, known, in the layer above interface 0
            rhs[rc] -= c_inc
            rhs[rf] -= eta[0] * (-1j * kyv[0]) * c_inc
    sol = np.linalg.solve(M, rhs)
    for m in range(L):
        A[m] = sol[ia(m)]
    for m in range(1, L + 1):
        B[m] = sol[ib(m)]
    return kx, kyv, A, B, c_inc


def incident(medium, theta: float, x, y) -> np.ndarray:
    k0 = float(np.asarray(medium.k)[0])
    x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    lay = layer_of(medium, y)
    u = np.exp(1j * (k0 * np.cos(theta) * x - k0 * np.sin(theta) * y))
    return np.where(lay == 0, u, 0.0)


def background(medium, theta: float, x, y) -> np.ndarray:
    x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    yint = np.asarray(medium.interfaces, dtype=np.float64).reshape(-1)
    L = yint.size
    kx, kyv, A, B, _ = background_coefficients(medium, theta)
    lay = layer_of(medium, y)
    out = np.zeros(np.broadcast(x, y).shape, dtype=np.complex128)
    for m in range(L + 1):
        sel = lay == m
        if not np.any(sel):
            continue
        ph = np.exp(1j * kx * x[sel])
        v = np.zeros(np.count_nonzero(sel), dtype=np.complex128)
        if m <= L - 1:
            v += A[m] * np.exp(1j * kyv[m] * (y[sel] - yint[m]))
        if m >= 1:
            v += B[m] * np.exp(-1j * kyv[m] * (y[sel] - yint[m - 1]))
        out[sel] = ph * v
    return out


def boundary_data(medium, theta: float, x, y) -> np.ndarray:
    """g = -(u_inc + u^b) on Gamma_0 and -u^b on deeper boundaries (eq. homogeneousscattering)."""
    return -(incident(medium, theta, x, y) + background(medium, theta, x, y))


def rhs(medium, theta: float, x, y) -> np.ndarray:
    """b = eta_{l'} g(c_{l'i}) (Sec. 3.3, eq. matrixandvec)."""
    eta = np.asarray(medium.eta, dtype=np.float64)
    return eta[layer_of(medium, y)] * boundary_data(medium, theta, x, y)
