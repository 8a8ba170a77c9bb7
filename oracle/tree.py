"""Plain quadtree, interaction lists and the domain-decomposition preconditioner.

TEST INFRASTRUCTURE ONLY.  This is a slow, loop-based reference of the tree
definition that the CUDA library implements, used to check the library's
integer outputs (permutation, boxes, lists) bit for bit, and a dense version
of the overlapping domain-decomposition preconditioner (Sec. 4.2).

Tree definition (the paper uses "the adaptive tree structure" of the FMM
framework without giving its parameters; this is the reading used here):
  * root square: centre of the points' bounding box, side
    W = max(extent) * (1 + 2^-10) (W = 1 for a single point);
  * coordinates quantised once to 20 bits: q = floor(((x - x0)/W) * 2^20),
    clamped to [0, 2^20 - 1]; the cell of a point at level l is q >> (20-l);
  * one box set per layer (the layer of a point is fixed by its height); all
    layers share the root square and the depth D, the smallest level at which
    no cell of any layer holds more than ``leaf_size`` points (at most 18);
  * points are ordered by (layer, Morton key at level D, original index);
    boxes by (level, layer, Morton key);
  * expansion order per level p_l = max(p, ceil(kR + 9 (kR)^(1/3))) with
    kR = k_max w_l / sqrt(2) (box radius times the largest wavenumber; the
    excess-bandwidth rule of wide-band multipole methods), w_l = W / 2^l, and
    expansions are used from the first level l0 >= 2 with p_l <= 80 (coarser
    levels only pass their lists down);
  * free-space lists (same layer): the candidates of box T are the children
    of its parent's near list (the root of T's layer at level 0); below l0
    all candidates stay near; from l0 on a candidate is near if its cell
    touches T's cell (Chebyshev offset <= 1), otherwise it is in T's M2L list;
    the near list at level D is the leaf's P2P list;
  * reaction lists, one set per non-zero component (l, *, l', star) of
    Sec. 3.1 (the remark on zero components): source boxes of layer l and
    target boxes of layer l'; the image-frame vertical offset of a box pair is
    D = h_*(S) + h_star(T) + H_c: heights above/below the interface each wave
    last met of the reaction expansion centres, plus the thickness of the
    layers the wave must cross (the effective transmission distance of
    Sec. 3.2).  A box's reaction expansion centre is its cell centre, moved
    for a cell that straddles that interface to the middle of the part of the
    cell on the layer's side (cell bounds lo = y0 + iy w, hi = y0 + (iy+1) w);
    a candidate is far (M2L) if D >= 2 w_l (1 - 1e-9), or if its cell column
    differs from T's by at least 2 while |k_y(T')| (w_l - D) <= 16, with
    T' = k_max + 0.75 (where the moment tables' contour leaves the real axis)
    and k_y = sqrt(T'^2 - k^2) for the smaller wavenumber of the two layers;
    otherwise near.  (The second bound keeps the spectral integrand of the
    pair's moment table bounded; the paper's admissibility by the effective
    distance alone does not say how far apart horizontally separated boxes
    must be.)
"""

from __future__ import annotations

import math

import numpy as np

QBITS = 20
D_CAP = 18
P_CAP = 80
COND_EXP = 16.0   # bound on log of the moment-table integrand growth of column-separated pairs
L0_MIN = 2


def layer_of(interfaces, y):
    yint = np.asarray(interfaces, dtype=np.float64).reshape(-1)
    y = np.asarray(y, dtype=np.float64)
    return np.sum(y[:, None] < yint[None, :], axis=1).astype(np.int64)


def morton(ix: int, iy: int, level: int) -> int:
    key = 0
    for b in range(level):
        key |= ((ix >> b) & 1) << (2 * b)
        key |= ((iy >> b) & 1) << (2 * b + 1)
    return key


def components(L: int):
    """Non-zero reaction components in library order: (ls, s_arrive, lt, t_depart), 0 = up, 1 = down."""
    out = []
    for ls in range(L + 1):
        for a in (0, 1):
            if a == 0 and ls >= L:
                continue
            if a == 1 and ls <= 0:
                continue
            for lt in range(L + 1):
                for b in (0, 1):
                    if b == 0 and lt <= 0:
                        continue
                    if b == 1 and lt >= L:
                        continue
                    out.append((ls, a, lt, b))
    return out


def comp_extra_thickness(yint, comp) -> float:
    """H_c: total thickness of the layers the reflected/transmitted wave must cross."""
    ls, a, lt, b = comp
    H = lambda m: yint[m - 1] - yint[m]
    if ls == lt:
        return H(ls) if a == b else 0.0
    if ls < lt:
        h = sum(H(m) for m in range(ls + 1, lt))
        if a == 1:
            h += H(ls)
        if b == 1:
            h += H(lt)
        return h
    h = sum(H(m) for m in range(lt + 1, ls))
    if a == 0:
        h += H(ls)
    if b == 0:
        h += H(lt)
    return h


def src_height(yint, ls, a, y):
    return (y - yint[ls]) if a == 0 else (yint[ls - 1] - y)


def tgt_height(yint, lt, b, y):
    return (yint[lt - 1] - y) if b == 0 else (y - yint[lt])


def clipped_height(y_if, above, lo, hi):
    """Height above (or below) the interface y_if of the centre of the part of the
    cell [lo, hi] that lies on the valid side (the side holding the layer's points)."""
    if above:
        return 0.5 * (max(lo, y_if) + hi) - y_if
    return y_if - 0.5 * (lo + min(hi, y_if))


def src_height_box(yint, ls, a, lo, hi):
    # arrival up: heights above the layer's bottom interface; down: below its top one
    return clipped_height(yint[ls], True, lo, hi) if a == 0 else clipped_height(yint[ls - 1], False, lo, hi)


def tgt_height_box(yint, lt, b, lo, hi):
    # departure up: depth below the layer's top interface; down: height above its bottom one
    return clipped_height(yint[lt - 1], False, lo, hi) if b == 0 else clipped_height(yint[lt], True, lo, hi)


class Tree:
    def __init__(self, pts, interfaces, k, p: int = 20, leaf_size: int = 64):
        pts = np.asarray(pts, dtype=np.float64)
        self.yint = [float(v) for v in np.asarray(interfaces, dtype=np.float64).reshape(-1)]
        self.L = len(self.yint)
        self.n = pts.shape[0]
        self.layer = layer_of(self.yint, pts[:, 1])
        self.k = [float(v) for v in np.asarray(k, dtype=np.float64).reshape(-1)]
        xmin, xmax = float(pts[:, 0].min()), float(pts[:, 0].max())
        ymin, ymax = float(pts[:, 1].min()), float(pts[:, 1].max())
        ext = max(xmax - xmin, ymax - ymin)
        W = ext * (1.0 + 1.0 / 1024.0) if ext > 0 else 1.0
        cx, cy = 0.5 * (xmin + xmax), 0.5 * (ymin + ymax)
        self.W, self.x0, self.y0 = W, cx - 0.5 * W, cy - 0.5 * W
        scale = float(1 << QBITS)
        qx = np.floor(((pts[:, 0] - self.x0) / W) * scale).astype(np.int64)
        qy = np.floor(((pts[:, 1] - self.y0) / W) * scale).astype(np.int64)
        self.qx = np.clip(qx, 0, (1 << QBITS) - 1)
        self.qy = np.clip(qy, 0, (1 << QBITS) - 1)
        # depth
        D = D_CAP
        for l in range(0, D_CAP + 1):
            sh = QBITS - l
            counts = {}
            ok = True
            for i in range(self.n):
                key = (int(self.layer[i]), int(self.qx[i] >> sh), int(self.qy[i] >> sh))
                counts[key] = counts.get(key, 0) + 1
                if counts[key] > leaf_size:
                    ok = False
                    break
            if ok:
                D = l
                break
        self.D = D
        kmax = float(np.max(k))
        self.p_level = []
        for l in range(D + 1):
            kr = kmax * (W / float(1 << l)) * 0.70710678118654752
            self.p_level.append(max(p, int(math.ceil(kr + 9.0 * math.pow(kr, 1.0 / 3.0)))))
        self.l0 = D + 1
        for l in range(L0_MIN, D + 1):
            if self.p_level[l] <= P_CAP:
                self.l0 = l
                break
        # sort points
        sh = QBITS - D
        keys = [(int(self.layer[i]), morton(int(self.qx[i] >> sh), int(self.qy[i] >> sh), D), i)
                for i in range(self.n)]
        keys.sort()
        self.perm = np.array([t[2] for t in keys], dtype=np.int64)
        # boxes
        self.box_level, self.box_layer, self.box_ix, self.box_iy = [], [], [], []
        self.box_begin, self.box_end, self.box_parent = [], [], []
        self.level_start = []
        index = {}
        for l in range(D + 1):
            self.level_start.append(len(self.box_level))
            shl = QBITS - l
            cur = None
            for pos in range(self.n):
                i = self.perm[pos]
                cell = (int(self.layer[i]), int(self.qx[i] >> shl), int(self.qy[i] >> shl))
                if cell != cur:
                    # boxes are in (layer, Morton) order because the point order is
                    b = len(self.box_level)
                    index[(l,) + cell] = b
                    self.box_level.append(l)
                    self.box_layer.append(cell[0])
                    self.box_ix.append(cell[1])
                    self.box_iy.append(cell[2])
                    self.box_begin.append(pos)
                    self.box_end.append(pos + 1)
                    self.box_parent.append(-1 if l == 0 else index[(l - 1, cell[0], cell[1] >> 1, cell[2] >> 1)])
                    cur = cell
                else:
                    self.box_end[-1] = pos + 1
        self.level_start.append(len(self.box_level))
        nb = len(self.box_level)
        self.nbox = nb
        self.children = [[] for _ in range(nb)]
        for b in range(nb):
            if self.box_parent[b] >= 0:
                self.children[self.box_parent[b]].append(b)
        self.comps = components(self.L)
        self._free_lists()
        self._reaction_lists()

    # -- geometry helpers ------------------------------------------------------
    def width(self, l):
        return self.W / float(1 << l)

    def centre(self, b):
        w = self.width(self.box_level[b])
        return (self.x0 + (self.box_ix[b] + 0.5) * w, self.y0 + (self.box_iy[b] + 0.5) * w)

    def boxes_at(self, l, layer=None):
        r = range(self.level_start[l], self.level_start[l + 1])
        return [b for b in r if layer is None or self.box_layer[b] == layer]

    # -- lists -------------------------------------------------------------------
    def _free_lists(self):
        nb = self.nbox
        near = [[] for _ in range(nb)]
        self.V_free = [[] for _ in range(nb)]
        for l in range(self.D + 1):
            for T in self.boxes_at(l):
                if l == 0:
                    cands = [T]
                else:
                    cands = [c for S in near[self.box_parent[T]] for c in self.children[S]]
                for S in sorted(cands):
                    if l < self.l0:
                        near[T].append(S)
                    elif abs(self.box_ix[S] - self.box_ix[T]) <= 1 and abs(self.box_iy[S] - self.box_iy[T]) <= 1:
                        near[T].append(S)
                    else:
                        self.V_free[T].append(S)
        self.U_free = {T: near[T] for T in self.boxes_at(self.D)}

    def cell_y(self, b):
        w = self.width(self.box_level[b])
        return self.y0 + self.box_iy[b] * w, self.y0 + (self.box_iy[b] + 1) * w

    def comp_D(self, c, S, T):
        ls, a, lt, b = self.comps[c]
        loS, hiS = self.cell_y(S)
        loT, hiT = self.cell_y(T)
        return (src_height_box(self.yint, ls, a, loS, hiS) + tgt_height_box(self.yint, lt, b, loT, hiT)) + \
            comp_extra_thickness(self.yint, self.comps[c])

    def _reaction_lists(self):
        # A pair that only the column offset separates is admitted while the spectral
        # integrand of its moment table stays bounded: on the real stretch of the
        # contour, up to T' = k_max + 0.75, the expansions' vertical extent (at most
        # w / 2 on either side) against the effective distance D lets it grow like
        # exp(|k_y(T')| (w - D)), k_y for the smaller of the two layers' wavenumbers.
        # The bound exp(16) keeps the cancellation in the tables far below the
        # truncation error; larger growth (wide-band cells with D << w) lost up to
        # 3e-5 of an entry in the four-layer medium k = 6, 10, 8, 12.
        self.V_react = []
        self.U_react = []
        t_tab = max(self.k) + 0.75
        for c, (ls, a, lt, b) in enumerate(self.comps):
            kl = min(self.k[ls], self.k[lt])
            ky_tab = math.sqrt(t_tab * t_tab - kl * kl)
            near = {}
            V = {}
            for l in range(self.D + 1):
                w = self.width(l)
                for T in self.boxes_at(l, lt):
                    if l == 0:
                        cands = self.boxes_at(0, ls)
                    else:
                        cands = [ch for S in near[self.box_parent[T]] for ch in self.children[S]]
                    nl, vl = [], []
                    for S in sorted(cands):
                        if l < self.l0:
                            nl.append(S)
                            continue
                        Dc = self.comp_D(c, S, T)
                        far = (abs(self.box_ix[S] - self.box_ix[T]) >= 2 and ky_tab * (w - Dc) <= COND_EXP) or \
                            Dc >= 2.0 * w * (1.0 - 1e-9)
                        (vl if far else nl).append(S)
                    near[T] = nl
                    if vl:
                        V[T] = vl
            self.V_react.append(V)
            self.U_react.append({T: near[T] for T in self.boxes_at(self.D, lt)})


def dd_preconditioner_dense(tree: Tree, pts, w, k, is_diag) -> np.ndarray:
    """Dense matrix of the restricted overlapping DD preconditioner (Sec. 4.2).

    For every leaf B of every layer: J = points of B and of its same-layer
    neighbour leaves (the leaf's free-space near list), P_B the free-space
    Nystrom block on J with the self terms I^s on the diagonal (eq. localmatix),
    and the rows of P_B^{-1} that belong to B's points are scattered into P^{-1}.
    """
    from .nystrom import free_block

    pts = np.asarray(pts, dtype=np.float64)
    n = pts.shape[0]
    Pinv = np.zeros((n, n), dtype=np.complex128)
    for B in tree.boxes_at(tree.D):
        lay = tree.box_layer[B]
        J = []
        for S in tree.U_free[B]:
            J.extend(tree.perm[tree.box_begin[S]:tree.box_end[S]].tolist())
        J = np.array(J, dtype=np.int64)
        own = tree.perm[tree.box_begin[B]:tree.box_end[B]]
        P = free_block(k[lay], pts[J], pts[J], w[J], exclude_self=True)
        P[np.arange(J.size), np.arange(J.size)] = is_diag[J]
        Pi = np.linalg.inv(P)
        pos = {int(j): a for a, j in enumerate(J)}
        rows = np.array([pos[int(i)] for i in own], dtype=np.int64)
        Pinv[np.ix_(own, J)] = Pi[rows, :]
    return Pinv
