"""The quadtree and every interaction list as the library builds them on the GPU
(csrc/tree_gpu.cu), against the oracle's tree (oracle/tree.py) bit for bit: root square,
depth, orders, point order, boxes of every level, free-space near/far lists and the
reaction lists of every component, at full workload sizes (65,536 points in three layers;
1,048,576 points in four layers, 150k boxes, 36 components) and on the wide-band cases
whose coarse cells straddle the interfaces."""

import numpy as np
import pytest

from oracle import nystrom as onys
from oracle import tree as otree
from tests.test_tree_host import _compare
from workloads import config_c2, config_c3, config_c4, layered_wide, layered_wide_c3

pytestmark = pytest.mark.gpu

LISTS = ["perm", "p_level", "box_level", "box_layer", "box_ix", "box_iy", "box_begin", "box_end", "box_parent",
         "vfree_ptr", "vfree_idx", "ufree_ptr", "ufree_idx", "vreact_ptr", "vreact_idx", "vreact_comp",
         "ureact_ptr", "ureact_idx", "ureact_comp"]


def _gpu_tree(lf, wl, pts, w, p, leaf):
    med = wl.medium
    M = lf.medium_create(med.interfaces, med.k, med.eta)
    G = lf.geometry_build(M, pts, w, p=p, leaf_size=leaf)
    q = lambda nm: lf.geometry_query(G, nm)
    tp = lf.geometry_query(G, "tree_params", np.float64)
    yint = np.asarray(med.interfaces, dtype=np.float64)
    h = dict(x0=tp[0], y0=tp[1], W=tp[2], D=int(tp[3]), l0=int(tp[4]),
             comps=[tuple(int(v) for v in c) for c in q("components").reshape(-1, 4)],
             layer_in=np.sum(pts[:, 1][:, None] < yint[None, :], axis=1))
    for nm in LISTS:
        h[nm] = q(nm)
    G.destroy()
    return h


@pytest.mark.parametrize("case", ["c2", "c3", "c4_four_layers", "wide_p20_leaf8", "wide_p6_leaf3", "wide_c3"])
def test_gpu_tree_and_lists_bit_exact(gpu_lib, case):
    if case == "c2":
        wl, p, leaf = config_c2(), 20, 64
    elif case == "c3":
        wl, p, leaf = config_c3(), 20, 64
    elif case == "c4_four_layers":
        wl = next(w for w in config_c4() if w.medium.n_layers == 4)
        p, leaf = wl.p, wl.leaf_size
    elif case == "wide_p20_leaf8":
        wl, p, leaf = layered_wide(), 20, 8
    elif case == "wide_p6_leaf3":
        wl, p, leaf = layered_wide(), 6, 3
    else:
        wl, p, leaf = layered_wide_c3(), 20, 8
    pts, w, _, _ = onys.elements(wl.bodies)
    h = _gpu_tree(gpu_lib, wl, pts, w, p, leaf)
    T = otree.Tree(pts, wl.medium.interfaces, wl.medium.k, p=p, leaf_size=leaf)
    assert T.nbox == len(h["box_level"])
    _compare(h, T)
