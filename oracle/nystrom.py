"""Lowest-order Nystrom discretisation, plain dense form (Sec. 3.3).

Test infrastructure only: used by tests/, the smoke check and bench.py's CPU
baseline; the library never imports or calls it.

Boundaries are split into straight elements (chords between consecutive
polygon vertices); the density is constant on each element and collocated at
the element centre, read as the chord midpoint with weight |Gamma_e| = chord
length (eq. linearSystem).  Matrix entries (eq. matrixelmemts):

  K[i, e] = |Gamma_e| G_{l_e l_i}(c_e, c_i)                  e != i
  K[i, i] = |Gamma_i| G^r_{l_i l_i}(c_i, c_i) + I^s_i

with the analytic self term (eq. ApproximateComputation)

  I^s_i = [ i/4 - (1/(2 pi)) (gamma + ln(k |Gamma_i| / 4) - 1) ] |Gamma_i|.

Rows are collocation points (layer l'), columns elements (layer l); the
unknown is Phi = eta phi and the right-hand side b = eta g (eq. matrixandvec).
The scattered field follows the representation (eq. integralrep)

  u^s(r) = (1/eta_{l(r)}) sum_e Phi_e |Gamma_e| G_{l_e l(r)}(c_e, r).
"""

from __future__ import annotations

import numpy as np

from . import core
from .green import gf, layer_of

EULER_GAMMA = 0.57721566490153286060651209008240243


def elements(bodies):
    """Chord midpoints, chord lengths, outward unit normals and body ids of CCW polygons."""
    pts, w, nrm, bid = [], [], [], []
    for b, v in enumerate(bodies):
        v = np.asarray(v, dtype=np.float64)
        v2 = np.roll(v, -1, axis=0)
        t = v2 - v
        ln = np.hypot(t[:, 0], t[:, 1])
        pts.append(0.5 * (v + v2))
        w.append(ln)
        nrm.append(np.stack([t[:, 1], -t[:, 0]], axis=1) / ln[:, None])
        bid.append(np.full(v.shape[0], b, dtype=np.int64))
    return (np.concatenate(pts), np.concatenate(w), np.concatenate(nrm), np.concatenate(bid))


def self_term(k, w) -> np.ndarray:
    """I^s = [i/4 - (1/2pi)(gamma + ln(k w/4) - 1)] w."""
    w = np.asarray(w, dtype=np.float64)
    return (0.25j - (EULER_GAMMA + np.log(np.asarray(k) * w / 4.0) - 1.0) / (2.0 * np.pi)) * w


def free_block(k: float, pts_t, pts_s, w_s, exclude_self: bool) -> np.ndarray:
    """|Gamma_e| (i/4) H_0(k |c_e - c_i|) for rows i in pts_t, columns e in pts_s."""
    dx = pts_t[:, None, 0] - pts_s[None, :, 0]
    dy = pts_t[:, None, 1] - pts_s[None, :, 1]
    r = np.hypot(dx, dy)
    if exclude_self:
        r = np.where(r == 0.0, 1.0, r)
    out = gf(k, r) * w_s[None, :]
    if exclude_self:
        out[np.hypot(dx, dy) == 0.0] = 0.0
    return out


def dense_matrix(medium, pts, w, tol_rel: float = 1e-13, reaction: bool = True) -> np.ndarray:
    """The dense Nystrom matrix K (N x N, complex128)."""
    pts = np.asarray(pts, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n = pts.shape[0]
    lay = layer_of(medium, pts[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    K = np.zeros((n, n), dtype=np.complex128)
    # free-space part: same layer, e != i
    for l in np.unique(lay):
        idx = np.flatnonzero(lay == l)
        blk = free_block(k[l], pts[idx], pts[idx], w[idx], exclude_self=True)
        K[np.ix_(idx, idx)] = blk
    # reaction part: all pairs, including e == i; G^r(field = c_e, source = c_i)
    if reaction and np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], pts[:, 0], pts[:, 1], tol_rel=tol_rel)
        K += Gr.T * w[None, :]
    # analytic self term
    K[np.arange(n), np.arange(n)] += self_term(k[lay], w)
    return K


def dense_rows(medium, pts, w, rows, tol_rel: float = 1e-13) -> np.ndarray:
    """Selected full rows of K (for sampled checks at sizes too large for the dense matrix)."""
    pts = np.asarray(pts, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    lay = layer_of(medium, pts[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    out = np.zeros((rows.size, pts.shape[0]), dtype=np.complex128)
    for a, i in enumerate(rows):
        same = np.flatnonzero(lay == lay[i])
        r = np.hypot(pts[same, 0] - pts[i, 0], pts[same, 1] - pts[i, 1])
        v = np.zeros(same.size, dtype=np.complex128)
        nz = r > 0
        v[nz] = gf(k[lay[i]], r[nz]) * w[same[nz]]
        out[a, same] = v
    if np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], pts[rows, 0], pts[rows, 1], tol_rel=tol_rel)
        out += Gr.T * w[None, :]
    out[np.arange(rows.size), rows] += self_term(k[lay[rows]], w[rows])
    return out


def dense_row_block(medium, pts, w, row: int, cols, tol_rel: float = 1e-13) -> np.ndarray:
    """Entries K[row, cols] of one row (a bounded sample of the dense definition)."""
    pts = np.asarray(pts, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    cols = np.asarray(cols, dtype=np.int64)
    lay = layer_of(medium, pts[:, 1])
    k = np.asarray(medium.k, dtype=np.float64)
    out = np.zeros(cols.size, dtype=np.complex128)
    same = lay[cols] == lay[row]
    r = np.hypot(pts[cols, 0] - pts[row, 0], pts[cols, 1] - pts[row, 1])
    sel = same & (r > 0)
    out[sel] = gf(k[lay[row]], r[sel]) * w[cols[sel]]
    if np.asarray(medium.interfaces).size > 0:
        g = core.gr_block(medium, pts[cols, 0], pts[cols, 1], pts[row:row + 1, 0], pts[row:row + 1, 1],
                          tol_rel=tol_rel)
        out += g[:, 0] * w[cols]
    out[cols == row] += self_term(k[lay[row]], w[row])
    return out


def field(medium, pts, w, Phi, targets, tol_rel: float = 1e-13) -> np.ndarray:
    """Scattered field u^s at off-boundary targets from the unknown Phi = eta phi."""
    pts = np.asarray(pts, dtype=np.float64)
    targets = np.asarray(targets, dtype=np.float64).reshape(-1, 2)
    w = np.asarray(w, dtype=np.float64)
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
            r = np.hypot(targets[ti, None, 0] - pts[None, si, 0], targets[ti, None, 1] - pts[None, si, 1])
            u[ti] += gf(k[l], r) @ q[si]
    if np.asarray(medium.interfaces).size > 0:
        Gr = core.gr_block(medium, pts[:, 0], pts[:, 1], targets[:, 0], targets[:, 1], tol_rel=tol_rel)
        u += Gr.T @ q
    return u / eta[lay_t]
