"""Layered Green's function, plain definition (Sec. 3.1, eqs. layeredGreensfun, freegreensfun).

Test infrastructure only: used by tests/, the smoke check and bench.py's CPU
baseline; the library never imports or calls it.

G_{ll'}(r, r') = delta_{ll'} (i/4) H_0^(1)(k_l |r - r'|) + G^r_{ll'}(r, r')

r = (x, y) is the field point (layer l), r' = (xs, ys) the source point
(layer l').  G^r comes from oracle_core.c (direct interface solve + contour
quadrature).  H_0^(1) is scipy's Hankel function (AMOS), pinned in the tests
against its power series, the large-argument asymptotics and the Wronskian.
"""

from __future__ import annotations

import numpy as np
from scipy.special import hankel1

from . import core


def layer_of(medium, y) -> np.ndarray:
    """Layer index of height(s) y: layer l is  -d_l < y < -d_{l-1}  (Sec. 2.1)."""
    y = np.asarray(y, dtype=np.float64)
    yint = np.asarray(medium.interfaces, dtype=np.float64).reshape(-1)
    return np.sum(y[..., None] < yint, axis=-1).astype(np.int64)


def gf(k: float, r) -> np.ndarray:
    """Free-space kernel (i/4) H_0^(1)(k r)."""
    return 0.25j * hankel1(0, k * np.asarray(r, dtype=np.float64))


def G(medium, x, y, xs, ys, tol_rel: float = 1e-13) -> np.ndarray:
    """Full layered Green's function for arrays of (field, source) pairs."""
    x, y, xs, ys = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (x, y, xs, ys)))
    lf, ls = layer_of(medium, y), layer_of(medium, ys)
    out = core.gr_pairs(medium, x, y, xs, ys, tol_rel=tol_rel).reshape(x.shape)
    same = lf == ls
    if np.any(same):
        k = np.asarray(medium.k, dtype=np.float64)[lf[same]]
        out[same] += gf(k, np.hypot(x[same] - xs[same], y[same] - ys[same]))
    return out


def gr_spectral(medium, lam, y: float, ys: float) -> np.ndarray:
    """Spectral reaction field Gt^r(lambda; y, ys) from the direct interface solve.

    Sum of the four amplitudes times e^{i k_{l,y} h(y)} e^{i k_{l',y} h(ys)}, with
    the heights measured from the interface each wave last met (the field
    point's bottom interface for an up-going arrival, its top interface for a
    down-going one; likewise at the source).
    """
    lam = np.atleast_1d(np.asarray(lam, dtype=np.complex128))
    yint = np.asarray(medium.interfaces, dtype=np.float64).reshape(-1)
    L = yint.size
    k = np.asarray(medium.k, dtype=np.float64)
    lf = int(layer_of(medium, y))
    ls = int(layer_of(medium, ys))
    S = core.spectral_amp(medium, lf, ls, lam)

    def ky(kk):
        s = np.sqrt(kk ** 2 - lam ** 2)
        return np.where(s.imag < 0, -s, s)

    kf, ks = ky(k[lf]), ky(k[ls])
    ef_up = np.exp(1j * kf * (y - yint[lf])) if lf <= L - 1 else 0.0
    ef_dn = np.exp(1j * kf * (yint[lf - 1] - y)) if lf >= 1 else 0.0
    es_up = np.exp(1j * ks * (yint[ls - 1] - ys)) if ls >= 1 else 0.0
    es_dn = np.exp(1j * ks * (ys - yint[ls])) if ls <= L - 1 else 0.0
    return (S[:, 0] * ef_up * es_up + S[:, 1] * ef_up * es_dn
            + S[:, 2] * ef_dn * es_up + S[:, 3] * ef_dn * es_dn)
