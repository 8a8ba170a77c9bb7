"""The library's host tree builder (csrc/tree.cpp) against the oracle's tree, bit for
bit, at full workload sizes on the CPU: points, boxes, orders, free-space and reaction
interaction lists.  tests/tree_harness.cpp drives build_tree from a file."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import nystrom as onys
from oracle import tree as otree
from workloads import config_c2, config_c4, layered_wide

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_build")   # git-ignored
CSRC = os.path.join(ROOT, "paper_2511_12450_gb300", "csrc")

ARRAYS = ["perm", "layer_sorted", "p_level", "box_level", "box_layer", "box_ix", "box_iy", "box_begin",
          "box_end", "box_parent", "vfree_ptr", "vfree_idx", "ufree_ptr", "ufree_idx", "vreact_ptr",
          "vreact_idx", "vreact_comp", "ureact_ptr", "ureact_idx", "ureact_comp"]


def _cuda_include():
    for d in [os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"]:
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def harness():
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    os.makedirs(WORK, exist_ok=True)
    exe = os.path.join(WORK, "tree_harness")
    cmd = [cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-I", inc, "-I", CSRC, os.path.join(ROOT, "tests", "tree_harness.cpp"),
           os.path.join(CSRC, "tree.cpp"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def _run(exe, pts, med, p, leaf, tag):
    n, nl = pts.shape[0], med.n_layers
    yint = np.asarray(med.interfaces, dtype=np.float64)
    # layer = number of interfaces above the point (interfaces decrease downwards)
    layer = np.sum(pts[:, 1][:, None] < yint[None, :], axis=1).astype(np.int32)
    src = os.path.join(WORK, f"tree_in_{tag}.bin")
    dst = os.path.join(WORK, f"tree_out_{tag}.bin")
    with open(src, "wb") as f:
        f.write(np.array([n, nl, p, leaf], dtype=np.int32).tobytes())
        f.write(yint.tobytes())
        f.write(np.asarray(med.k, dtype=np.float64).tobytes())
        f.write(np.asarray(med.eta, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(pts[:, 0]).tobytes())
        f.write(np.ascontiguousarray(pts[:, 1]).tobytes())
        f.write(layer.tobytes())
    res = subprocess.run([exe, src, dst], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr
    buf = open(dst, "rb").read()
    os.unlink(src)
    os.unlink(dst)
    off = 0
    geo = np.frombuffer(buf, np.float64, 3, off); off += 24
    D, l0, nc = np.frombuffer(buf, np.int32, 3, off); off += 12
    comps = np.frombuffer(buf, np.int32, 4 * nc, off).reshape(-1, 4); off += 16 * nc
    out = dict(x0=geo[0], y0=geo[1], W=geo[2], D=int(D), l0=int(l0), comps=[tuple(int(v) for v in c) for c in comps],
               layer_in=layer)
    for name in ARRAYS:
        m = int(np.frombuffer(buf, np.int64, 1, off)[0]); off += 8
        out[name] = np.frombuffer(buf, np.int32, m, off).copy(); off += 4 * m
    assert off == len(buf)
    return out


def _compare(h, T):
    assert np.array_equal(h["layer_in"], np.asarray(T.layer))
    assert (h["x0"], h["y0"], h["W"], h["D"], h["l0"]) == (T.x0, T.y0, T.W, T.D, T.l0)
    assert np.array_equal(h["perm"], np.asarray(T.perm))
    assert np.array_equal(h["p_level"], np.asarray(T.p_level))
    for nm in ["box_level", "box_layer", "box_ix", "box_iy", "box_begin", "box_end", "box_parent"]:
        assert np.array_equal(h[nm], np.asarray(getattr(T, nm))), nm
    assert h["comps"] == T.comps
    vp, vi = h["vfree_ptr"], h["vfree_idx"]
    for b in range(T.nbox):
        assert list(vi[vp[b]:vp[b + 1]]) == T.V_free[b], b
    up, ui = h["ufree_ptr"], h["ufree_idx"]
    for b in T.boxes_at(T.D):
        assert list(ui[up[b]:up[b + 1]]) == T.U_free[b], b
    rp, ri, rc = h["vreact_ptr"], h["vreact_idx"], h["vreact_comp"]
    for b in range(T.nbox):
        got = {}
        for e in range(rp[b], rp[b + 1]):
            got.setdefault(int(rc[e]), []).append(int(ri[e]))
        want = {c: T.V_react[c][b] for c in range(len(T.comps)) if b in T.V_react[c]}
        assert got == want, b
    urp, uri, urc = h["ureact_ptr"], h["ureact_idx"], h["ureact_comp"]
    for b in T.boxes_at(T.D):
        got = {}
        for e in range(urp[b], urp[b + 1]):
            got.setdefault(int(urc[e]), []).append(int(uri[e]))
        want = {c: T.U_react[c][b] for c in range(len(T.comps)) if T.U_react[c].get(b)}
        assert got == want, b


def test_c2_full_size_tree_is_bit_exact(harness):
    # N = 65,536 in three layers, 64 bodies, bodies straddling both interfaces
    wl = config_c2()
    pts, _, _, _ = onys.elements(wl.bodies)
    h = _run(harness, pts, wl.medium, wl.p, wl.leaf_size, "c2")
    T = otree.Tree(pts, wl.medium.interfaces, wl.medium.k, p=wl.p, leaf_size=wl.leaf_size)
    assert T.nbox == len(h["box_level"]) and T.D == 9 and len(T.comps) == 16
    _compare(h, T)


def test_four_layer_and_wide_band_trees_are_bit_exact(harness):
    # a four-layer medium with k up to 12 (the largest C4 geometry's stack), and the
    # wide-band case whose coarse levels raise the order and straddle interfaces
    wl4 = next(w for w in config_c4() if w.medium.n_layers == 4)
    pts4, _, _, _ = onys.elements(wl4.bodies)
    T4 = otree.Tree(pts4, wl4.medium.interfaces, wl4.medium.k, p=wl4.p, leaf_size=wl4.leaf_size)
    _compare(_run(harness, pts4, wl4.medium, wl4.p, wl4.leaf_size, "c4"), T4)
    ww = layered_wide()
    ptsw, _, _, _ = onys.elements(ww.bodies)
    for p, leaf in [(20, 8), (6, 3)]:
        Tw = otree.Tree(ptsw, ww.medium.interfaces, ww.medium.k, p=p, leaf_size=leaf)
        _compare(_run(harness, ptsw, ww.medium, p, leaf, f"wide{p}"), Tw)


def test_largest_workload_tree_is_bit_exact(harness):
    # the precision form's workload: N = 1,048,576 in four layers (k up to 12), 150k boxes,
    # depth 11, expansions from level 4 (order 75) down to order 20, 36 reaction components
    from workloads import config_c3

    wl = config_c3()
    pts, _, _, _ = onys.elements(wl.bodies)
    h = _run(harness, pts, wl.medium, wl.p, wl.leaf_size, "c3")
    T = otree.Tree(pts, wl.medium.interfaces, wl.medium.k, p=wl.p, leaf_size=wl.leaf_size)
    assert pts.shape[0] == 1 << 20 and T.D == 11 and T.l0 == 4 and len(T.comps) == 36
    _compare(h, T)
