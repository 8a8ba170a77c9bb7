"""Thin ctypes binding of the C ABI in include/lfmm.h (argument marshalling only).

Every function here has the name of the C entry point without the ``lfmm_``
prefix and does nothing but check/convert arguments and call the library:
all computation happens in the CUDA library.  Vectors may be numpy arrays
(host memory) or CUDA torch tensors (device memory, passed with
LFMM_DEVICE_PTRS on the current torch stream).  Complex vectors are
complex128, column-major [n x nrhs] (a 1-D array is one column).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblfmm.so")

LFMM_OK = 0
LFMM_NOT_CONVERGED = 1
LFMM_ERR_INVALID_ARG = -1
LFMM_ERR_OUT_OF_MEMORY = -2
LFMM_ERR_CUDA = -3
LFMM_ERR_NODE_ON_INTERFACE = -4
LFMM_ERR_QUADRATURE = -5
LFMM_ERR_TIMEOUT = -6
LFMM_ERR_HBM_BUDGET = -7
LFMM_DEVICE_PTRS = 1
LFMM_MIXED = 2
LFMM_PROFILE_STAGES = 1
LFMM_AUTOTUNE = 2
LFMM_COMBINED_FIELD = 4
LFMM_SIMT_M2L = 8
LFMM_C64 = 16
STAGES = ["p2m", "m2m", "m2l", "l2l", "l2p", "near", "gather", "scatter"]

EXPORTED = [
    "lfmm_medium_create", "lfmm_medium_destroy", "lfmm_geometry_build", "lfmm_geometry_destroy",
    "lfmm_rhs_plane_wave", "lfmm_matvec", "lfmm_gmres_solve", "lfmm_eval_field",
    "lfmm_polygon_elements", "lfmm_geometry_query", "lfmm_last_error", "lfmm_matvec_static",
    "lfmm_precond_apply", "lfmm_matvec_batch",
    "lfmm_server_create", "lfmm_server_submit", "lfmm_server_wait", "lfmm_server_stats", "lfmm_server_destroy",
]


class LfmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lfmm status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("leaf_size", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GmresParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precision", ctypes.c_int32)]


class GmresInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("solve_seconds", ctypes.c_double),
                ("refinements", ctypes.c_int32), ("fp64_matvecs", ctypes.c_int32), ("op_rel_diff", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved", ctypes.c_int32), ("hbm_budget", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("p", ctypes.c_int32),
                ("interface_y", ctypes.c_void_p), ("wavenumber", ctypes.c_void_p), ("density", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("points", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("angle_rad", ctypes.c_double), ("tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("normals", ctypes.c_void_p), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("queue_seconds", ctypes.c_double), ("service_seconds", ctypes.c_double),
                ("latency_seconds", ctypes.c_double), ("setup_seconds", ctypes.c_double),
                ("footprint_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None


def library():
    """Load the compiled library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
        lib.lfmm_medium_create.argtypes = [i32, dp, dp, dp, ctypes.POINTER(vp)]
        lib.lfmm_medium_destroy.argtypes = [vp]
        lib.lfmm_geometry_build.argtypes = [vp, i64, dp, dp, dp, ctypes.POINTER(Params), ctypes.POINTER(vp)]
        lib.lfmm_geometry_destroy.argtypes = [vp]
        lib.lfmm_rhs_plane_wave.argtypes = [vp, i32, dp, vp, i32, vp]
        lib.lfmm_matvec.argtypes = [vp, i32, vp, vp, i32, vp]
        lib.lfmm_matvec_static.argtypes = [vp, vp, vp, vp]
        lib.lfmm_precond_apply.argtypes = [vp, i32, vp, vp, i32, vp]
        lib.lfmm_matvec_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(vp),
                                          ctypes.POINTER(vp), i32, vp]
        lib.lfmm_gmres_solve.argtypes = [vp, i32, vp, vp, ctypes.POINTER(GmresParams), ctypes.POINTER(GmresInfo), vp]
        lib.lfmm_eval_field.argtypes = [vp, i32, vp, i64, dp, vp, i32, vp]
        lib.lfmm_polygon_elements.argtypes = [i32, ctypes.POINTER(ctypes.c_int32), dp, dp, dp, dp]
        lib.lfmm_geometry_query.argtypes = [vp, ctypes.c_char_p, vp, i64, ctypes.POINTER(i64)]
        lib.lfmm_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(vp)]
        lib.lfmm_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(i64)]
        lib.lfmm_server_wait.argtypes = [vp, i64, vp, ctypes.POINTER(GmresInfo), ctypes.POINTER(RequestTimes)]
        lib.lfmm_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
        lib.lfmm_server_destroy.argtypes = [vp]
        lib.lfmm_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name != "lfmm_last_error":
                getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _check(status: int):
    if status < 0:
        raise LfmmError(status, library().lfmm_last_error().decode())
    return status


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _stream_of(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Medium:
    def __init__(self, handle, interfaces, k, eta):
        self.handle = handle
        self.interfaces, self.k, self.eta = interfaces, k, eta

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.lfmm_medium_destroy(self.handle)
            self.handle = None


class Geometry:
    def __init__(self, handle, medium: Medium, n: int):
        self.handle = handle
        self.medium = medium   # keeps the medium alive
        self.n = n

    def destroy(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.lfmm_geometry_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.destroy()


def medium_create(interfaces, k, eta) -> Medium:
    yint = _f64(interfaces).reshape(-1)
    kk = np.asarray(k)
    kc = np.ascontiguousarray(kk.astype(np.complex128).reshape(-1))
    et = _f64(eta).reshape(-1)
    h = ctypes.c_void_p()
    _check(library().lfmm_medium_create(int(kc.size), _dp(yint) if yint.size else None,
                                        _dp(kc.view(np.float64)), _dp(et), ctypes.byref(h)))
    return Medium(h, yint, kc, et)


def geometry_build(medium: Medium, points, weights, normals=None, p: int = 20, leaf_size: int = 64,
                   profile: bool = False, autotune: bool = False, combined: bool = False) -> Geometry:
    """Tree, tables, near field and preconditioner for the elements (points, weights).

    combined=True builds the combined-field operator 1/2 I + D - i k S (second kind;
    needs the outward unit normals) instead of the paper's single layer."""
    pts = _f64(points).reshape(-1, 2)
    w = _f64(weights).reshape(-1)
    nrm = _f64(normals).reshape(-1, 2) if normals is not None else None
    flags = ((LFMM_PROFILE_STAGES if profile else 0) | (LFMM_AUTOTUNE if autotune else 0)
             | (LFMM_COMBINED_FIELD if combined else 0))
    prm = Params(int(p), int(leaf_size), flags, 0)
    h = ctypes.c_void_p()
    _check(library().lfmm_geometry_build(medium.handle, pts.shape[0], _dp(pts), _dp(w),
                                         _dp(nrm) if nrm is not None else None, ctypes.byref(prm),
                                         ctypes.byref(h)))
    return Geometry(h, medium, pts.shape[0])


def _vec_args(v, n, allow_c64=True):
    """(pointer, nrhs, flags, keepalive) for a complex vector argument; complex64
    vectors (where the call takes them) add LFMM_C64 to the flags."""
    if _is_torch_cuda(v):
        import torch

        c64 = v.dtype == torch.complex64
        if not (v.dtype == torch.complex128 or (c64 and allow_c64)) or not v.is_contiguous():
            raise TypeError("contiguous complex128 tensor expected" + (" (or complex64)" if allow_c64 else ""))
        return ctypes.c_void_p(v.data_ptr()), v.numel() // n, LFMM_DEVICE_PTRS | (LFMM_C64 if c64 else 0), v
    a = np.asarray(v)
    c64 = a.dtype == np.complex64
    if not (a.dtype == np.complex128 or (c64 and allow_c64)):
        raise TypeError("complex128 expected" + (" (or complex64)" if allow_c64 else ""))
    if not a.flags["F_CONTIGUOUS" if a.ndim == 2 else "C_CONTIGUOUS"]:
        raise ValueError("vector must be column-major contiguous")
    return ctypes.c_void_p(a.ctypes.data), a.size // n, LFMM_C64 if c64 else 0, a


def _empty_like(v, n, nrhs):
    if _is_torch_cuda(v):
        import torch

        return torch.empty((n,) if nrhs == 1 else (nrhs, n), dtype=v.dtype, device=v.device)
    dt = np.asarray(v).dtype
    return np.zeros(n, dtype=dt) if nrhs == 1 else np.zeros((n, nrhs), dtype=dt, order="F")


def rhs_plane_wave(g: Geometry, angles_rad, out=None, stream=None, device=False, single=False):
    """b for plane waves at the given angles; single=True returns complex64 (LFMM_C64)."""
    ang = _f64(angles_rad).reshape(-1)
    nrhs = ang.size
    if out is None:
        if device:
            import torch

            out = torch.empty((nrhs, g.n) if nrhs > 1 else (g.n,),
                              dtype=torch.complex64 if single else torch.complex128, device="cuda")
        else:
            out = _empty_like(np.zeros(1, np.complex64 if single else np.complex128), g.n, nrhs)
    ptr, _, flags, keep = _vec_args(out, g.n)
    st = _stream_of(stream) if flags & LFMM_DEVICE_PTRS else ctypes.c_void_p(0)
    _check(library().lfmm_rhs_plane_wave(g.handle, nrhs, _dp(ang), ptr, flags, st))
    return out


def matvec(g: Geometry, x, y=None, stream=None, mixed: bool = False, simt_m2l: bool = False):
    """y = K x.  mixed=True applies the precision form (FP32 far field; its M2L on the
    tensor cores for 16 or more columns unless simt_m2l=True)."""
    xp, nrhs, flags, keep = _vec_args(x, g.n)
    if y is None:
        y = _empty_like(x, g.n, nrhs)
    yp, _, flags_y, keep_y = _vec_args(y, g.n)
    if flags != flags_y:
        raise ValueError("x and y must both be host arrays or both device tensors, of one complex dtype")
    st = _stream_of(stream) if flags & LFMM_DEVICE_PTRS else ctypes.c_void_p(0)
    flags |= (LFMM_MIXED if mixed else 0) | (LFMM_SIMT_M2L if simt_m2l else 0)
    _check(library().lfmm_matvec(g.handle, nrhs, xp, yp, flags, st))
    return y


def matvec_batch(geos, xs, ys=None, stream=None):
    """y_i = K_i x_i for several geometries in shared launches (CUDA tensors, all complex128
    or all complex64; each [n_i] or [nrhs_i, n_i] as in matvec)."""
    geos = list(geos)
    xs = list(xs)
    if len(geos) != len(xs) or not geos:
        raise ValueError("one x per geometry expected")
    if ys is None:
        ys = [_empty_like(x, g.n, _vec_args(x, g.n)[1]) for g, x in zip(geos, xs)]
    ys = list(ys)
    args = [(_vec_args(x, g.n), _vec_args(y, g.n)) for g, x, y in zip(geos, xs, ys)]
    flags = {a[0][2] for a in args} | {a[1][2] for a in args}
    if len(flags) != 1 or not (next(iter(flags)) & LFMM_DEVICE_PTRS):
        raise TypeError("matvec_batch takes CUDA tensors of one complex dtype")
    n = len(geos)
    hv = (ctypes.c_void_p * n)(*[g.handle for g in geos])
    nr = (ctypes.c_int32 * n)(*[a[0][1] for a in args])
    xp = (ctypes.c_void_p * n)(*[a[0][0] for a in args])
    yp = (ctypes.c_void_p * n)(*[a[1][0] for a in args])
    _check(library().lfmm_matvec_batch(n, hv, nr, xp, yp, next(iter(flags)), _stream_of(stream)))
    return ys


def precond_apply(g: Geometry, x, y=None, stream=None):
    """y = P^{-1} x, the overlapping domain-decomposition preconditioner (Sec. 4.2) alone."""
    xp, nrhs, flags, keep = _vec_args(x, g.n, allow_c64=False)
    if y is None:
        y = _empty_like(x, g.n, nrhs)
    yp, _, flags_y, keep_y = _vec_args(y, g.n, allow_c64=False)
    if flags != flags_y:
        raise ValueError("x and y must both be host arrays or both device tensors")
    st = _stream_of(stream) if flags & LFMM_DEVICE_PTRS else ctypes.c_void_p(0)
    _check(library().lfmm_precond_apply(g.handle, nrhs, xp, yp, flags, st))
    return y


def matvec_static(g: Geometry, x, y, stream=None):
    """y = K x with the library's fixed device work array (device tensors, one column, no allocation)."""
    if not (_is_torch_cuda(x) and _is_torch_cuda(y)):
        raise TypeError("matvec_static takes CUDA tensors")
    # contiguous complex128 only: the library reads and writes 16 n bytes through these pointers
    xp, nx, fx, keep = _vec_args(x, g.n, allow_c64=False)
    yp, ny, fy, keep_y = _vec_args(y, g.n, allow_c64=False)
    if x.numel() != g.n or y.numel() != g.n:
        raise ValueError("one column of n entries expected")
    _check(library().lfmm_matvec_static(g.handle, xp, yp, _stream_of(stream)))
    return y


def gmres_solve(g: Geometry, b, x=None, tol: float = 1e-8, max_iter: int = 1000, precond: bool = True,
                stream=None, precision: int = 0, restart: int = 0):
    """GMRES to tol.  precision=1: iterative refinement with inner solves on the precision form.
    restart=m > 0: GMRES(m), each pass from the recomputed residual with at most m Krylov vectors."""
    bp, nrhs, flags, keep = _vec_args(b, g.n, allow_c64=False)
    if x is None:
        x = _empty_like(b, g.n, nrhs)
    xp, _, _, keep_x = _vec_args(x, g.n, allow_c64=False)
    prm = GmresParams(float(tol), int(max_iter), int(restart), 1 if precond else 0, int(precision))
    info = GmresInfo()
    st = _stream_of(stream) if flags else ctypes.c_void_p(0)
    status = _check(library().lfmm_gmres_solve(g.handle, nrhs, bp, xp, ctypes.byref(prm), ctypes.byref(info), st))
    d = info.as_dict()
    d["status"] = status
    return x, d


def eval_field(g: Geometry, density, targets, stream=None):
    dpp, nrhs, flags, keep = _vec_args(density, g.n)
    tg = _f64(targets).reshape(-1, 2)
    m = tg.shape[0]
    dt = np.complex64 if flags & LFMM_C64 else np.complex128
    u = np.zeros(m, dtype=dt) if nrhs == 1 else np.zeros((m, nrhs), dtype=dt, order="F")
    st = _stream_of(stream) if flags & LFMM_DEVICE_PTRS else ctypes.c_void_p(0)
    _check(library().lfmm_eval_field(g.handle, nrhs, dpp, m, _dp(tg), ctypes.c_void_p(u.ctypes.data), flags, st))
    return u


def polygon_elements(polygons):
    polys = [_f64(p).reshape(-1, 2) for p in polygons]
    counts = np.array([p.shape[0] for p in polys], dtype=np.int32)
    verts = np.ascontiguousarray(np.concatenate(polys, axis=0))
    n = int(counts.sum())
    pts = np.zeros((n, 2))
    w = np.zeros(n)
    nrm = np.zeros((n, 2))
    _check(library().lfmm_polygon_elements(len(polys), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           _dp(verts), _dp(pts), _dp(w), _dp(nrm)))
    return pts, w, nrm


def geometry_query(g: Geometry, name: str, dtype=np.int32) -> np.ndarray:
    need = ctypes.c_int64(0)
    _check(library().lfmm_geometry_query(g.handle, name.encode(), None, 0, ctypes.byref(need)))
    out = np.zeros(need.value // np.dtype(dtype).itemsize, dtype=dtype)
    _check(library().lfmm_geometry_query(g.handle, name.encode(), ctypes.c_void_p(out.ctypes.data), need.value,
                                         ctypes.byref(need)))
    return out


def tuning(g: Geometry) -> dict:
    """The M2L work-item schedule of a geometry and, when it was built with
    autotune=True, the measured milliseconds of one FP64 M2L with the default and
    the chosen schedule."""
    v = geometry_query(g, "tuning", np.float64)
    return {"item_work": int(v[0]), "wide_rows": bool(v[1]), "ms_default": float(v[2]), "ms_best": float(v[3])}


def stage_times(g: Geometry) -> dict:
    """Per-stage launch counts and total milliseconds (geometries built with profile=True)."""
    v = geometry_query(g, "stage_times", np.float64).reshape(-1, 2)
    return {name: {"count": int(v[i, 0]), "ms": float(v[i, 1])} for i, name in enumerate(STAGES)}


class Server:
    """Request loop for scattering solves (lfmm_server_*): ``slots`` concurrent requests,
    admission by estimated device footprint within ``hbm_budget`` bytes."""

    def __init__(self, slots: int, hbm_budget: int):
        self.handle = ctypes.c_void_p()
        _check(library().lfmm_server_create(ctypes.byref(ServerParams(int(slots), 0, int(hbm_budget))),
                                            ctypes.byref(self.handle)))
        self._keep = {}

    def submit(self, interfaces, k, eta, points, weights, angle_rad: float, tol: float = 1e-8,
               precision: int = 0, p: int = 20, leaf_size: int = 64, max_iter: int = 1000,
               precond: bool = True, normals=None, combined: bool = False) -> int:
        """Queue a scattering solve; combined=True solves with the combined-field
        operator (needs the outward unit normals)."""
        yint = _f64(interfaces).reshape(-1)
        kc = np.ascontiguousarray(np.asarray(k).astype(np.complex128).reshape(-1))
        et = _f64(eta).reshape(-1)
        pts = _f64(points).reshape(-1, 2)
        w = _f64(weights).reshape(-1)
        req = Request(int(kc.size), int(p), ctypes.c_void_p(yint.ctypes.data) if yint.size else None,
                      ctypes.c_void_p(kc.ctypes.data), ctypes.c_void_p(et.ctypes.data), int(w.size),
                      ctypes.c_void_p(pts.ctypes.data), ctypes.c_void_p(w.ctypes.data), float(angle_rad),
                      float(tol), int(precision), int(leaf_size), int(max_iter), 1 if precond else 0)
        nrm = _f64(normals).reshape(-1, 2) if normals is not None else None
        if nrm is not None:
            req.normals = ctypes.c_void_p(nrm.ctypes.data)
        req.flags = LFMM_COMBINED_FIELD if combined else 0
        t = ctypes.c_int64(0)
        _check(library().lfmm_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = w.size
        return t.value

    def wait(self, ticket: int):
        n = self._keep.pop(ticket)
        x = np.empty(n, dtype=np.complex128)
        info, times = GmresInfo(), RequestTimes()
        st = _check(library().lfmm_server_wait(self.handle, int(ticket), ctypes.c_void_p(x.ctypes.data),
                                               ctypes.byref(info), ctypes.byref(times)))
        d = info.as_dict()
        d["status"] = st
        return x, d, times.as_dict()

    def stats(self):
        b, r = ctypes.c_int64(0), ctypes.c_int32(0)
        _check(library().lfmm_server_stats(self.handle, ctypes.byref(b), ctypes.byref(r)))
        return {"peak_bytes": b.value, "peak_running": r.value}

    def close(self):
        if self.handle:
            library().lfmm_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
