"""Combined-field variant of the Nystrom operator, plain dense form.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves the first-kind single-layer equation (Sec. 3.3).  This module
is the opt-in second-kind alternative: the scattered field is represented by a
double- plus single-layer potential with the layered Green's function,

  u^s(r) = (1/eta_{l(r)}) sum_e Phi_e |Gamma_e| [ n_e . grad_{c_e} - i kappa_e ] G_{l_e l(r)}(c_e, r),

where n_e is the element's outward unit normal, kappa_e = k_{l(e)} the
wavenumber of its layer, and G_{l l'}(c_e, r) the layered Green's function of
Sec. 3.1 with c_e in the field slot (the slot the single-layer matrix of
eq. matrixelmemts integrates over).  Differentiating with respect to that point
is differentiating the potential of a source on the element, so every term
satisfies the transmission conditions; the free-space part carries the classical
jump of the double layer, +1/2 phi on the exterior side, and the reaction part
is smooth there.  Collocated at the element centres and scaled by eta like the
single-layer system (Phi = eta phi, b = eta g):

  K^cf[i, e] = |Gamma_e| [ n_e . grad_{c_e} - i kappa_e ] G_{l_e l_i}(c_e, c_i)          e != i
  K^cf[i, i] = 1/2 + |Gamma_i| n_i . grad_1 G^r(c_i, c_i) - i kappa_i (|Gamma_i| G^r(c_i, c_i) + I^s_i)

The free-space double layer of a straight element on its own centre vanishes
(n . (c_i - y) = 0 on the segment); I^s is the single-layer self term of
eq. ApproximateComputation.  The right-hand side is unchanged.
"""

from __future__ import annotations

import numpy as np
from scipy.special import hankel1

from . import core
from .green import gf, layer_of
from .nystrom import self_term


def grad_free(k: float, pf, ps):
    """Gradient of (i/4) H_0(k |r - r_s|) with respect to the field point r, for
    field points pf (rows) and source points ps (columns): (d/dx, d/dy).  Pairs at
    zero distance give 0 (the principal value over a straight element)."""
    dx = pf[:, None, 0] - ps[None, :, 0]
    dy = pf[:, None, 1] - ps[None, :, 1]
    r = np.hypot(dx, dy)
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    # d/dr (i/4) H_0(k r) = -(i/4) k H_1(k r)
    d = -0.25j * k * hankel1(1, k * rs)
    gx = np.where(zero, 0.0, d * dx / rs)
    gy = np.where(zero, 0.0, d * dy / rs)
    return gx, gy


def dense_matrix_cf(medium, pts, w, nrm, tol_rel: float = 1e-13) -> np.ndarray:
    """The dense combined-field matrix K^cf (N x N, complex128)."""
    pts = np.asarray(pts, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    n = pts.shape[0]
    lay = layer_of(medium, pts[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    kap = k[lay]
    K = np.zeros((n, n), dtype=np.complex128)
    # free space, same layer: rows i (targets), columns e; the field slot is c_e
    for l in np.unique(lay):
        idx = np.flatnonzero(lay == l)
        p = pts[idx]
        gx, gy = grad_free(k[l], p, p)          # [e, i]: field c_e, source c_i
        r = np.hypot(p[:, None, 0] - p[None, :, 0], p[:, None, 1] - p[None, :, 1])
        g = np.where(r == 0.0, 0.0, gf(k[l], np.where(r == 0.0, 1.0, r)))
        ker = nrm[idx, 0, None] * gx + nrm[idx, 1, None] * gy - 1j * k[l] * g   # [e, i]
        K[np.ix_(idx, idx)] = (ker * w[idx, None]).T
    if np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], pts[:, 0], pts[:, 1], tol_rel=tol_rel)
        gx, gy = core.gr_grad_block(medium, pts[:, 0], pts[:, 1], pts[:, 0], pts[:, 1], tol_rel=tol_rel)
        ker = nrm[:, 0, None] * gx + nrm[:, 1, None] * gy - 1j * kap[:, None] * Gr   # [e, i]
        K += ker.T * w[None, :]
    K[np.arange(n), np.arange(n)] += 0.5 - 1j * kap * self_term(kap, w)
    return K


def dense_rows_cf(medium, pts, w, nrm, rows, tol_rel: float = 1e-13) -> np.ndarray:
    """Selected full rows of K^cf (sampled checks at sizes too large for the dense matrix)."""
    pts = np.asarray(pts, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    lay = layer_of(medium, pts[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    kap = k[lay]
    out = np.zeros((rows.size, pts.shape[0]), dtype=np.complex128)
    for a, i in enumerate(rows):
        same = np.flatnonzero(lay == lay[i])
        gx, gy = grad_free(k[lay[i]], pts[same], pts[i:i + 1])
        r = np.hypot(pts[same, 0] - pts[i, 0], pts[same, 1] - pts[i, 1])
        g = np.where(r == 0.0, 0.0, gf(k[lay[i]], np.where(r == 0.0, 1.0, r)))
        out[a, same] = (nrm[same, 0] * gx[:, 0] + nrm[same, 1] * gy[:, 0] - 1j * k[lay[i]] * g) * w[same]
    if np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], pts[rows, 0], pts[rows, 1], tol_rel=tol_rel)
        gx, gy = core.gr_grad_block(medium, pts[:, 0], pts[:, 1], pts[rows, 0], pts[rows, 1], tol_rel=tol_rel)
        ker = nrm[:, 0, None] * gx + nrm[:, 1, None] * gy - 1j * kap[:, None] * Gr
        out += ker.T * w[None, :]
    out[np.arange(rows.size), rows] += 0.5 - 1j * kap[rows] * self_term(kap[rows], w[rows])
    return out


def field_cf(medium, pts, w, nrm, Phi, targets, tol_rel: float = 1e-13) -> np.ndarray:
    """Scattered field of the combined-field representation at off-boundary targets."""
    pts = np.asarray(pts, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    Phi = np.asarray(Phi, dtype=np.complex128)
    lay_s = layer_of(medium, pts[:, 1])
    lay_t = layer_of(medium, targets[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    eta = np.asarray(medium.eta, dtype=np.float64)
    q = Phi * w
    u = np.zeros(targets.shape[0], dtype=np.complex128)
    for l in np.unique(lay_t):
        ti = np.flatnonzero(lay_t == l)
        si = np.flatnonzero(lay_s == l)
        if si.size:
            gx, gy = grad_free(k[l], pts[si], targets[ti])            # [e, t]
            r = np.hypot(pts[si, None, 0] - targets[None, ti, 0], pts[si, None, 1] - targets[None, ti, 1])
            ker = nrm[si, 0, None] * gx + nrm[si, 1, None] * gy - 1j * k[l] * gf(k[l], r)
            u[ti] += ker.T @ q[si]
    if np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], targets[:, 0], targets[:, 1], tol_rel=tol_rel)
        gx, gy = core.gr_grad_block(medium, pts[:, 0], pts[:, 1], targets[:, 0], targets[:, 1], tol_rel=tol_rel)
        ker = nrm[:, 0, None] * gx + nrm[:, 1, None] * gy - 1j * k[lay_s][:, None] * Gr
        u += ker.T @ q
    return u / eta[lay_t]
