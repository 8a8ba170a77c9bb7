"""C-ABI checks that need no GPU: the library loads and exports every declared symbol;
host-only helpers and argument validation."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lfmm.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"\b(lfmm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_12450_gb300 import _build, lfmm

    _build.build()
    return lfmm


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lfmm_matvec" in names and "lfmm_gmres_solve" in names
    so = lib.library()
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib.EXPORTED)


def test_polygon_elements_host_helper(lib):
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=float)
    pts, w, nrm = lib.polygon_elements([sq])
    np.testing.assert_allclose(pts, [[0.5, 0], [1, 0.5], [0.5, 1], [0, 0.5]])
    np.testing.assert_allclose(w, [1, 1, 1, 1])
    np.testing.assert_allclose(nrm, [[0, -1], [1, 0], [0, 1], [-1, 0]])
    with pytest.raises(lib.LfmmError):
        lib.polygon_elements([np.array([[0, 0], [0, 0], [1, 1]], dtype=float)])


def test_medium_validation(lib):
    m = lib.medium_create([0.0, -2.0], [4.0, 6.0, 8.0], [1.0, 2.0, 3.0])
    assert m.handle
    for bad in [
        dict(interfaces=[0.0, 1.0], k=[1, 2, 3], eta=[1, 1, 1]),       # not decreasing
        dict(interfaces=[0.0], k=[1.0, -2.0], eta=[1, 1]),             # k <= 0
        dict(interfaces=[0.0], k=[1.0, 2.0 + 0.1j], eta=[1, 1]),       # complex k unsupported
        dict(interfaces=[0.0], k=[1.0, 2.0], eta=[1, 0.0]),            # eta <= 0
    ]:
        with pytest.raises(lib.LfmmError) as ei:
            lib.medium_create(**bad)
        assert ei.value.status == lib.LFMM_ERR_INVALID_ARG


def test_geometry_argument_validation_before_device_work(lib):
    # every check of lfmm_geometry_build runs on the host before any device call,
    # so these need no GPU
    m = lib.medium_create([0.0, -2.0], [4.0, 6.0, 8.0], [1.0, 2.0, 3.0])
    good = np.array([[0.1, 0.5], [0.3, -1.0]])
    w = np.array([0.1, 0.1])
    cases = [
        (np.zeros((0, 2)), np.zeros(0), {}, lib.LFMM_ERR_INVALID_ARG),                 # empty
        (good, np.array([0.1, -0.1]), {}, lib.LFMM_ERR_INVALID_ARG),                   # weight <= 0
        (np.array([[np.nan, 0.5], [0.3, -1.0]]), w, {}, lib.LFMM_ERR_INVALID_ARG),     # not finite
        (good, w, {"p": 0}, lib.LFMM_ERR_INVALID_ARG),                                 # order < 1
        (good, w, {"p": 81}, lib.LFMM_ERR_INVALID_ARG),                                # order > 80
        (good, w, {"leaf_size": 0}, lib.LFMM_ERR_INVALID_ARG),
        (good, w, {"leaf_size": 1025}, lib.LFMM_ERR_INVALID_ARG),
        (np.array([[0.1, 0.0], [0.3, -1.0]]), w, {}, lib.LFMM_ERR_NODE_ON_INTERFACE),  # on y = 0
        (np.array([[0.1, 0.5], [0.3, -2.0]]), w, {}, lib.LFMM_ERR_NODE_ON_INTERFACE),  # on y = -2
    ]
    for pts, ww, kw, code in cases:
        with pytest.raises(lib.LfmmError) as ei:
            lib.geometry_build(m, pts, ww, **kw)
        assert ei.value.status == code, (pts, kw)
    # the combined-field operator needs outward unit normals
    with pytest.raises(lib.LfmmError) as ei:
        lib.geometry_build(m, good, w, None, combined=True)
    assert ei.value.status == lib.LFMM_ERR_INVALID_ARG
    with pytest.raises(lib.LfmmError) as ei:
        lib.geometry_build(m, good, w, np.array([[1.0, 0.0], [0.6, 0.6]]), combined=True)
    assert ei.value.status == lib.LFMM_ERR_INVALID_ARG


def test_binding_constants_match_the_header(lib):
    with open(os.path.join(ROOT, "include", "lfmm.h")) as f:
        txt = f.read()
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(LFMM_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt))
    assert "LFMM_C64" in consts and "LFMM_DEVICE_PTRS" in consts
    for k, v in consts.items():
        if hasattr(lib, k):
            assert getattr(lib, k) == v, k
    missing = [k for k in consts if not hasattr(lib, k)]
    assert not missing, missing


def test_single_precision_vectors_marshal_with_the_c64_flag(lib):
    n = 8
    x = np.zeros(n, dtype=np.complex64)
    _, nrhs, flags, _ = lib._vec_args(x, n)
    assert nrhs == 1 and flags == lib.LFMM_C64
    X = np.zeros((n, 3), dtype=np.complex128, order="F")
    _, nrhs, flags, _ = lib._vec_args(X, n)
    assert nrhs == 3 and flags == 0
    with pytest.raises(TypeError):
        lib._vec_args(np.zeros(n, dtype=np.float64), n)

    class FakeGeometry:   # gmres_solve checks its vectors before calling the library
        n = 8
        handle = None

    with pytest.raises(TypeError):
        lib.gmres_solve(FakeGeometry(), x)


def test_failed_geometry_build_returns_a_null_handle(lib):
    import ctypes

    m = lib.medium_create([0.0], [4.0, 6.0], [1.0, 2.0])
    pts = np.array([[0.1, 0.0], [0.3, -1.0]])   # the first point lies on the interface
    w = np.array([0.1, 0.1])
    h = ctypes.c_void_p(12345)
    st = lib.library().lfmm_geometry_build(m.handle, 2, lib._dp(pts), lib._dp(w), None, None, ctypes.byref(h))
    assert st == lib.LFMM_ERR_NODE_ON_INTERFACE
    assert not h.value
    assert "interface" in lib.library().lfmm_last_error().decode()


def test_static_matvec_and_precond_reject_host_or_wrong_vectors_in_the_binding(lib):
    # the binding refuses what the device entry points would read out of bounds, before
    # any call into the library (no geometry or GPU needed)
    g = lib.Geometry(None, None, 8)
    x = np.zeros(8, dtype=np.complex128)
    with pytest.raises(TypeError):
        lib.matvec_static(g, x, np.zeros(8, dtype=np.complex128))   # host arrays
    with pytest.raises(TypeError):
        lib.precond_apply(g, x.astype(np.complex64))                # single precision


def test_null_arguments_rejected_by_every_vector_entry_point(lib):
    import ctypes

    so = lib.library()
    buf = (ctypes.c_double * 4)()
    assert so.lfmm_matvec_static(None, buf, buf, None) == lib.LFMM_ERR_INVALID_ARG
    assert "NULL" in so.lfmm_last_error().decode()
    assert so.lfmm_precond_apply(None, 1, buf, buf, 0, None) == lib.LFMM_ERR_INVALID_ARG
    assert so.lfmm_matvec(None, 1, buf, buf, 0, None) == lib.LFMM_ERR_INVALID_ARG
