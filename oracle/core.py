"""ctypes wrapper around oracle_core.c (test infrastructure only)."""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_spectral_amp.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_long, dp, dp]
        lib.oracle_gr_pairs.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp,
                                        ctypes.c_double, dp, ip]
        lib.oracle_gr_pairs_contour.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ip]
        lib.oracle_gr_block.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_long, dp, dp,
                                        ctypes.c_long, dp, dp, ctypes.c_double, dp]
        lib.oracle_gr_grad_block.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_long, dp, dp,
                                             ctypes.c_long, dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _medium_arrays(medium):
    yint = np.ascontiguousarray(np.asarray(medium.interfaces, dtype=np.float64).reshape(-1))
    k = np.ascontiguousarray(np.asarray(medium.k, dtype=np.float64).reshape(-1))
    eta = np.ascontiguousarray(np.asarray(medium.eta, dtype=np.float64).reshape(-1))
    if yint.size == 0:
        yint = np.zeros(1)
    return yint, k, eta


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def spectral_amp(medium, lf: int, ls: int, lam) -> np.ndarray:
    """Reaction amplitudes (4 per lambda) from the direct interface solve.

    Columns: (field up, source up), (field up, source down),
             (field down, source up), (field down, source down).
    """
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128).reshape(-1))
    yint, k, eta = _medium_arrays(medium)
    out = np.zeros((lam.size, 4), dtype=np.complex128)
    lam_ri = lam.view(np.float64)
    rc = _lib().oracle_spectral_amp(int(k.size), _dp(yint), _dp(k), _dp(eta), int(lf), int(ls),
                                    int(lam.size), _dp(lam_ri), _dp(out.view(np.float64)))
    if rc != 0:
        raise RuntimeError(f"oracle_spectral_amp failed ({rc})")
    return out


def gr_pairs(medium, x, y, xs, ys, tol_rel: float = 1e-13, check: bool = True) -> np.ndarray:
    """G^r((x,y), (xs,ys)) elementwise (field point first, source point second)."""
    x, y, xs, ys = (np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
                    for a in np.broadcast_arrays(x, y, xs, ys))
    n = x.size
    yint, k, eta = _medium_arrays(medium)
    out = np.zeros(n, dtype=np.complex128)
    st = np.zeros(n, dtype=np.int32)
    _lib().oracle_gr_pairs(int(k.size), _dp(yint), _dp(k), _dp(eta), n, _dp(x), _dp(y),
                           _dp(xs), _dp(ys), float(tol_rel), _dp(out.view(np.float64)),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if check and np.any(st != 0):
        bad = np.flatnonzero(st)
        raise RuntimeError(f"oracle G^r failed for {bad.size} pairs (status {np.unique(st[bad])})")
    return out


def gr_pairs_contour(medium, x, y, xs, ys, t_scale: float, h_scale: float, tol_rel: float = 1e-13) -> np.ndarray:
    """gr_pairs on a deformed contour: detour end T times t_scale (>= 1), depth h times
    h_scale (in (0, 1]).  The integral is contour independent (Cauchy), so this is a
    self-check of the contour and the quadrature, not a different quantity."""
    x, y, xs, ys = (np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
                    for a in np.broadcast_arrays(x, y, xs, ys))
    n = x.size
    yint, k, eta = _medium_arrays(medium)
    out = np.zeros(n, dtype=np.complex128)
    st = np.zeros(n, dtype=np.int32)
    rc = _lib().oracle_gr_pairs_contour(int(k.size), _dp(yint), _dp(k), _dp(eta), n, _dp(x), _dp(y),
                                        _dp(xs), _dp(ys), float(tol_rel), float(t_scale), float(h_scale),
                                        _dp(out.view(np.float64)), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise RuntimeError(f"oracle G^r on the scaled contour failed ({rc}, status {np.unique(st)})")
    return out


def gr_block(medium, xr, yr, xc, yc, tol_rel: float = 1e-13) -> np.ndarray:
    """Dense G^r block: rows are field points (xr,yr), columns source points (xc,yc)."""
    xr, yr, xc, yc = (np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
                      for a in (xr, yr, xc, yc))
    yint, k, eta = _medium_arrays(medium)
    out = np.zeros((xr.size, xc.size), dtype=np.complex128)
    rc = _lib().oracle_gr_block(int(k.size), _dp(yint), _dp(k), _dp(eta), xr.size, _dp(xr),
                                _dp(yr), xc.size, _dp(xc), _dp(yc), float(tol_rel),
                                _dp(out.view(np.float64)))
    if rc != 0:
        raise RuntimeError("oracle G^r block: quadrature or interface-solve failure")
    return out


def gr_grad_block(medium, xr, yr, xc, yc, tol_rel: float = 1e-13):
    """Gradient of G^r with respect to the FIELD point (xr, yr): two dense blocks
    (d/dx, d/dy), rows are field points, columns source points."""
    xr, yr, xc, yc = (np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
                      for a in (xr, yr, xc, yc))
    yint, k, eta = _medium_arrays(medium)
    gx = np.zeros((xr.size, xc.size), dtype=np.complex128)
    gy = np.zeros((xr.size, xc.size), dtype=np.complex128)
    rc = _lib().oracle_gr_grad_block(int(k.size), _dp(yint), _dp(k), _dp(eta), xr.size, _dp(xr),
                                     _dp(yr), xc.size, _dp(xc), _dp(yc), float(tol_rel),
                                     _dp(gx.view(np.float64)), _dp(gy.view(np.float64)))
    if rc != 0:
        raise RuntimeError("oracle grad G^r block: quadrature or interface-solve failure")
    return gx, gy
