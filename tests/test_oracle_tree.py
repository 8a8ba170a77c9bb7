"""Pins for the oracle's plain quadtree and interaction lists (brute force on small inputs).

Every (source, target) point pair of the free-space part (same layer) and of
every reaction component must be handled exactly once: either in the near
list of the target's leaf, or through exactly one M2L list entry between an
ancestor of the target and an ancestor of the source at the same level.
Every M2L entry must be well separated in the sense the expansions need.
"""

import numpy as np
import pytest

from oracle import tree
from oracle.nystrom import elements
from workloads import layered_small


@pytest.fixture(scope="module")
def small_tree():
    wl = layered_small(n_bodies=4, nodes=150, seed=11)
    pts, w, _, _ = elements(wl.bodies)
    T = tree.Tree(pts, wl.medium.interfaces, wl.medium.k, p=6, leaf_size=12)
    return T, pts


def _ancestors(T, leaf):
    out = {T.box_level[leaf]: leaf}
    b = leaf
    while T.box_parent[b] >= 0:
        b = T.box_parent[b]
        out[T.box_level[b]] = b
    return out


def test_points_and_boxes(small_tree):
    T, pts = small_tree
    assert sorted(T.perm.tolist()) == list(range(T.n))
    leaves = T.boxes_at(T.D)
    covered = np.zeros(T.n, dtype=int)
    for b in leaves:
        assert T.box_end[b] - T.box_begin[b] <= 12
        covered[T.box_begin[b]:T.box_end[b]] += 1
        lay = set(T.layer[T.perm[T.box_begin[b]:T.box_end[b]]].tolist())
        assert lay == {T.box_layer[b]}
    assert np.all(covered == 1)
    for b in range(T.nbox):
        if T.box_parent[b] >= 0:
            pb = T.box_parent[b]
            assert T.box_begin[pb] <= T.box_begin[b] and T.box_end[b] <= T.box_end[pb]
    assert T.l0 <= T.D, "test tree should exercise the far field"


def test_free_space_coverage(small_tree):
    T, pts = small_tree
    leaf_of = np.empty(T.n, dtype=int)
    for b in T.boxes_at(T.D):
        leaf_of[T.perm[T.box_begin[b]:T.box_end[b]]] = b
    anc = {b: _ancestors(T, b) for b in T.boxes_at(T.D)}
    Vset = {(t, s) for t in range(T.nbox) for s in T.V_free[t]}
    for i in range(T.n):
        for j in range(T.n):
            if T.layer[i] != T.layer[j]:
                continue
            ti, sj = leaf_of[i], leaf_of[j]
            hits = int(sj in T.U_free[ti])
            for l in range(T.l0, T.D + 1):
                if (anc[ti][l], anc[sj][l]) in Vset:
                    hits += 1
            assert hits == 1, (i, j)
    for t in range(T.nbox):
        for s in T.V_free[t]:
            assert max(abs(T.box_ix[s] - T.box_ix[t]), abs(T.box_iy[s] - T.box_iy[t])) >= 2
            assert t in T.V_free[s]


def test_reaction_coverage(small_tree):
    T, pts = small_tree
    leaf_of = np.empty(T.n, dtype=int)
    for b in T.boxes_at(T.D):
        leaf_of[T.perm[T.box_begin[b]:T.box_end[b]]] = b
    anc = {b: _ancestors(T, b) for b in T.boxes_at(T.D)}
    assert len(T.comps) == 4 * T.L * T.L
    n_far = 0
    for c, (ls, a, lt, b) in enumerate(T.comps):
        V = T.V_react[c]
        Vset = {(t, s) for t in V for s in V[t]}
        n_far += len(Vset)
        src = np.flatnonzero(T.layer == ls)
        tgt = np.flatnonzero(T.layer == lt)
        for i in tgt:
            for j in src:
                ti, sj = leaf_of[i], leaf_of[j]
                hits = int(sj in T.U_react[c].get(ti, []))
                for l in range(T.l0, T.D + 1):
                    if (anc[ti][l], anc[sj][l]) in Vset:
                        hits += 1
                assert hits == 1, (c, i, j)
        for t, lst in V.items():
            w = T.width(T.box_level[t])
            for s in lst:
                Dc = T.comp_D(c, s, t)
                assert abs(T.box_ix[s] - T.box_ix[t]) >= 2 or Dc >= 2 * w * (1 - 1e-9)
    assert n_far > 0
