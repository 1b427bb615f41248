"""Thin ctypes binding of libhps (include/hps.h): argument marshalling only.

Every entry point keeps the C name.  Host arrays are numpy float64 arrays;
device arrays are CUDA torch tensors (float64, contiguous), passed by pointer
when device_ptrs=True.  No step of the method runs here: a missing or unloadable
libhps.so raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhps.so"
_lib = None

HPS_OK = 0
HPS_EINVAL = -1
HPS_ENOMEM = -2
HPS_ESINGULAR = -3
HPS_ENOTCONVERGED = -4
HPS_EDEVICE = -5
HPS_FP64 = 0
HPS_MIXED = 1

COEFF_NAMES = ("c11", "c12", "c22", "c1", "c2", "c")

EXPORTS = ("hps_default_options", "hps_boundary_count", "hps_cheb_nodes",
           "hps_boundary_nodes_grid", "hps_build", "hps_boundary_nodes", "hps_solve",
           "hps_solve_ex", "hps_query", "hps_free", "hps_status_string", "hps_kernel_launches",
           "hps_profile_enable", "hps_profile_reset", "hps_profile_read", "hps_last_error",
           "hps_solve_static", "hps_build_batch", "hps_solve_batch", "hps_batch_size",
           "hps_estimate_bytes", "hps_release_workspace", "hps_dgemm_tc", "hps_apply_dtn",
           "hps_interpolate", "hps_sgemm_tc", "hps_leaf_residual", "hps_sinv_gj",
           # include/hps_serve.h
           "hps_server_default_options", "hps_server_create", "hps_server_destroy",
           "hps_server_submit_build", "hps_server_submit_solve", "hps_server_wait",
           "hps_server_result", "hps_server_release", "hps_server_release_operator",
           "hps_server_get_stats")


class HpsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        extra = lib().hps_last_error().decode() if status == HPS_EDEVICE else ""
        super().__init__(f"{where}: {lib().hps_status_string(status).decode()} ({status})"
                         + (f" [{extra}]" if extra else ""))


class Domain(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("fp64_top_levels", ctypes.c_int),
                ("device_ptrs", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("form_root_dtn", ctypes.c_int), ("refine_depth", ctypes.c_int),
                ("leaf_refine", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("d", Domain), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("p", ctypes.c_int),
                ("q", ctypes.c_int), ("c11", ctypes.c_void_p), ("c12", ctypes.c_void_p),
                ("c22", ctypes.c_void_p), ("c1", ctypes.c_void_p), ("c2", ctypes.c_void_p),
                ("c", ctypes.c_void_p)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("last_update", ctypes.c_double), ("bad_box", ctypes.c_int)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("workers", ctypes.c_int),
                ("max_rhs_per_solve", ctypes.c_int), ("device", ctypes.c_int)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("kind", ctypes.c_int), ("op", ctypes.c_int64),
                ("nrhs", ctypes.c_int), ("batch_rhs", ctypes.c_int), ("iterations", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "completed", "failed", "builds", "solves", "solve_calls", "rhs_solved",
        "resident_ops", "evicted_ops", "bytes_in_use", "peak_bytes_in_use", "budget")]


def lib():
    """Load libhps.so (built in-tree by paper_1307_2665_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"libhps.so not built ({_LIB_PATH}); run paper_1307_2665_gb300.build.build()")
    L = ctypes.CDLL(str(_LIB_PATH), mode=os.RTLD_LOCAL)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    L.hps_default_options.argtypes = [ctypes.POINTER(Options)]
    L.hps_default_options.restype = None
    L.hps_boundary_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hps_boundary_count.restype = ctypes.c_int64
    L.hps_cheb_nodes.argtypes = [Domain, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.hps_boundary_nodes_grid.argtypes = [Domain, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.hps_build.argtypes = [Domain, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            vp, vp, vp, vp, vp, vp, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.hps_boundary_nodes.argtypes = [vp, dp]
    L.hps_solve.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.POINTER(SolveInfo)]
    L.hps_solve_ex.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(SolveInfo)]
    L.hps_query.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64)]
    L.hps_free.argtypes = [vp]
    L.hps_kernel_launches.argtypes = []
    L.hps_kernel_launches.restype = ctypes.c_int64
    L.hps_profile_enable.argtypes = [ctypes.c_int]
    L.hps_profile_enable.restype = None
    L.hps_profile_reset.argtypes = []
    L.hps_profile_reset.restype = None
    L.hps_profile_read.argtypes = [ctypes.POINTER(KernelStat), ctypes.c_int]
    L.hps_profile_read.restype = ctypes.c_int
    L.hps_build_batch.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(Options),
                                  ctypes.POINTER(vp)]
    L.hps_build_batch.restype = ctypes.c_int
    L.hps_solve_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                  ctypes.POINTER(SolveInfo)]
    L.hps_solve_batch.restype = ctypes.c_int
    L.hps_batch_size.argtypes = [vp]
    L.hps_batch_size.restype = ctypes.c_int
    L.hps_solve_static.argtypes = [vp, vp, ctypes.c_int, vp]
    L.hps_solve_static.restype = ctypes.c_int
    L.hps_last_error.argtypes = []
    L.hps_last_error.restype = ctypes.c_char_p
    L.hps_status_string.argtypes = [ctypes.c_int]
    L.hps_status_string.restype = ctypes.c_char_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.hps_estimate_bytes.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(Options),
                                     ctypes.c_int, i64p, i64p, i64p]
    L.hps_release_workspace.argtypes = [vp]
    L.hps_dgemm_tc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp,
                               ctypes.c_int, vp, ctypes.c_int, ctypes.c_double, vp, ctypes.c_int]
    L.hps_dgemm_tc.restype = ctypes.c_int
    L.hps_sgemm_tc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp,
                               ctypes.c_int, vp, ctypes.c_int, ctypes.c_float, vp, ctypes.c_int]
    L.hps_sgemm_tc.restype = ctypes.c_int
    L.hps_leaf_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, vp, vp, vp, vp, ctypes.c_int, vp, vp,
                                    ctypes.c_int]
    L.hps_leaf_residual.restype = ctypes.c_int
    L.hps_sinv_gj.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
    L.hps_sinv_gj.restype = ctypes.c_int
    L.hps_apply_dtn.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int]
    L.hps_apply_dtn.restype = ctypes.c_int
    L.hps_interpolate.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int64, vp, ctypes.c_int]
    L.hps_interpolate.restype = ctypes.c_int
    L.hps_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
    L.hps_server_default_options.restype = None
    L.hps_server_create.argtypes = [ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)]
    L.hps_server_destroy.argtypes = [vp]
    L.hps_server_submit_build.argtypes = [vp, ctypes.POINTER(Problem), ctypes.POINTER(Options)]
    L.hps_server_submit_build.restype = ctypes.c_int64
    L.hps_server_submit_solve.argtypes = [vp, ctypes.c_int64, vp, ctypes.c_int]
    L.hps_server_submit_solve.restype = ctypes.c_int64
    L.hps_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(RequestInfo)]
    L.hps_server_result.argtypes = [vp, ctypes.c_int64, vp]
    L.hps_server_release.argtypes = [vp, ctypes.c_int64]
    L.hps_server_release_operator.argtypes = [vp, ctypes.c_int64]
    L.hps_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    for name in ("hps_estimate_bytes", "hps_release_workspace", "hps_server_create",
                 "hps_server_destroy", "hps_server_wait", "hps_server_result", "hps_server_release",
                 "hps_server_release_operator", "hps_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("hps_cheb_nodes", "hps_boundary_nodes_grid", "hps_build", "hps_boundary_nodes",
                 "hps_solve", "hps_solve_ex", "hps_query", "hps_free"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _domain(d):
    return Domain(*map(float, d))


def _ptr(a):
    """Pointer of a float64 numpy array or CUDA torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def default_options():
    o = Options()
    lib().hps_default_options(ctypes.byref(o))
    return o


def hps_boundary_count(nx, ny, q):
    return int(lib().hps_boundary_count(nx, ny, q))


def hps_cheb_nodes(domain, nx, ny, p):
    """(nx*ny, p, p, 2) coordinates of every leaf's Chebyshev grid."""
    xy = np.empty((nx * ny, p, p, 2))
    st = lib().hps_cheb_nodes(_domain(domain), nx, ny, p,
                              xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != HPS_OK:
        raise HpsError(st, "hps_cheb_nodes")
    return xy


def hps_boundary_nodes_grid(domain, nx, ny, q):
    """(nbnd, 2) coordinates of the Dirichlet nodes, in the order of f."""
    xy = np.empty((hps_boundary_count(nx, ny, q), 2))
    st = lib().hps_boundary_nodes_grid(_domain(domain), nx, ny, q,
                                       xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != HPS_OK:
        raise HpsError(st, "hps_boundary_nodes_grid")
    return xy


class Handle:
    """Owns an hps_handle; frees it on close() or garbage collection."""

    def __init__(self, ptr, domain, nx, ny, p, q, device_ptrs):
        self.ptr = ptr
        self.domain, self.nx, self.ny, self.p, self.q = domain, nx, ny, p, q
        self.device_ptrs = device_ptrs
        self.nbnd = hps_boundary_count(nx, ny, q)

    def close(self):
        if self.ptr:
            lib().hps_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _options(precision, device_ptrs, stream, refine_tol, max_refine, fp64_top_levels,
             form_root_dtn, refine_depth=None, leaf_refine=None):
    opt = default_options()
    opt.precision = precision
    opt.device_ptrs = 1 if device_ptrs else 0
    opt.stream = stream
    opt.form_root_dtn = 1 if form_root_dtn else 0
    if refine_tol is not None:
        opt.refine_tol = refine_tol
    if max_refine is not None:
        opt.max_refine = max_refine
    if fp64_top_levels is not None:
        opt.fp64_top_levels = fp64_top_levels
    if refine_depth is not None:
        opt.refine_depth = refine_depth
    if leaf_refine is not None:
        opt.leaf_refine = leaf_refine
    return opt


class BatchHandle:
    """Owns a batch hps_handle; frees it on close() or garbage collection."""

    def __init__(self, ptr, problems, device_ptrs):
        self.ptr = ptr
        self.problems = problems  # list of (domain, nx, ny, p, q)
        self.device_ptrs = device_ptrs

    def close(self):
        if self.ptr:
            lib().hps_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hps_build_batch(problems, precision=HPS_FP64, device_ptrs=False, stream=None,
                    refine_tol=None, max_refine=None, fp64_top_levels=None, form_root_dtn=False,
                    refine_depth=None, leaf_refine=None, check=True):
    """Batch build.  problems: list of dicts with keys domain, nx, ny, p, q, coeffs."""
    opt = _options(precision, device_ptrs, stream, refine_tol, max_refine, fp64_top_levels,
                   form_root_dtn, refine_depth, leaf_refine)
    arr = (Problem * len(problems))()
    for i, pr in enumerate(problems):
        arr[i].d = _domain(pr["domain"])
        arr[i].nx, arr[i].ny, arr[i].p, arr[i].q = pr["nx"], pr["ny"], pr["p"], pr["q"]
        for k in COEFF_NAMES:
            setattr(arr[i], k, _ptr(pr["coeffs"].get(k)))
    out = ctypes.c_void_p()
    st = lib().hps_build_batch(arr, len(problems), ctypes.byref(opt), ctypes.byref(out))
    if st != HPS_OK:
        if check:
            raise HpsError(st, "hps_build_batch")
        return st
    return BatchHandle(out.value, [(pr["domain"], pr["nx"], pr["ny"], pr["p"], pr["q"])
                                   for pr in problems], device_ptrs)


def hps_solve_batch(h: BatchHandle, fs, us, info=None, check=True):
    """Batch solve: fs[k] of shape (nrhs, nbnd_k), us[k] of shape (nrhs, nl_k, p_k, p_k)."""
    nrhs = fs[0].shape[0]
    fa = (ctypes.c_void_p * len(fs))(*[_ptr(f) for f in fs])
    ua = (ctypes.c_void_p * len(us))(*[_ptr(u) for u in us])
    inf = SolveInfo() if info is None else info
    st = lib().hps_solve_batch(h.ptr, fa, nrhs, ua, ctypes.byref(inf))
    inf.status = st
    if st != HPS_OK and check:
        raise HpsError(st, "hps_solve_batch")
    return us


def hps_build(domain, nx, ny, p, q, coeffs, precision=HPS_FP64, device_ptrs=False, stream=None,
              refine_tol=None, max_refine=None, fp64_top_levels=None, form_root_dtn=False,
              refine_depth=None, leaf_refine=None, check=True):
    """Build stage.  coeffs: dict name -> array of nx*ny*p*p values (or None).
    Returns a Handle, or raises HpsError (returns the status when check=False)."""
    opt = _options(precision, device_ptrs, stream, refine_tol, max_refine, fp64_top_levels,
                   form_root_dtn, refine_depth, leaf_refine)
    arrs = [coeffs.get(k) for k in COEFF_NAMES]
    out = ctypes.c_void_p()
    st = lib().hps_build(_domain(domain), nx, ny, p, q, *[_ptr(a) for a in arrs],
                         ctypes.byref(opt), ctypes.byref(out))
    if st != HPS_OK:
        if check:
            raise HpsError(st, "hps_build")
        return st
    return Handle(out.value, domain, nx, ny, p, q, device_ptrs)


def hps_boundary_nodes(h: Handle):
    xy = np.empty((h.nbnd, 2))
    st = lib().hps_boundary_nodes(h.ptr, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != HPS_OK:
        raise HpsError(st, "hps_boundary_nodes")
    return xy


def hps_solve(h: Handle, f, u=None, device_ptrs=None, info=None, check=True):
    """Solve stage.  f: (nrhs, nbnd) or (nbnd,) float64; u: output of shape
    (nrhs, nx*ny, p, p) (allocated on the host when omitted and f is on the host)."""
    dev = h.device_ptrs if device_ptrs is None else bool(device_ptrs)
    nrhs = 1 if f.ndim == 1 else f.shape[0]
    if u is None:
        if dev:
            raise ValueError("device solves need a preallocated u")
        u = np.empty((nrhs, h.nx * h.ny, h.p, h.p))
    inf = SolveInfo() if info is None else info
    st = lib().hps_solve_ex(h.ptr, _ptr(f), nrhs, _ptr(u), 1 if dev else 0, ctypes.byref(inf))
    inf.status = st
    if st != HPS_OK and check:
        raise HpsError(st, "hps_solve")
    return u


def hps_apply_dtn(h: Handle, f, g=None, device_ptrs=None, check=True):
    """g = T^1 f (the root DtN of a handle built with form_root_dtn=True).
    f: (nrhs, nbnd) or (nbnd,) float64; g: same shape (allocated on the host
    when omitted and f is on the host)."""
    dev = h.device_ptrs if device_ptrs is None else bool(device_ptrs)
    nrhs = 1 if f.ndim == 1 else f.shape[0]
    if g is None:
        if dev:
            raise ValueError("device applies need a preallocated g")
        g = np.empty(f.shape)
    st = lib().hps_apply_dtn(h.ptr, _ptr(f), nrhs, _ptr(g), 1 if dev else 0)
    if st != HPS_OK and check:
        raise HpsError(st, "hps_apply_dtn")
    return g if check else (g, st)


def hps_interpolate(h: Handle, u, xy, out=None, device_ptrs=None, check=True):
    """Solutions u (nrhs, nx*ny, p, p) evaluated at points xy (npts, 2):
    returns out (nrhs, npts)."""
    dev = h.device_ptrs if device_ptrs is None else bool(device_ptrs)
    nrhs = u.shape[0]
    npts = xy.shape[0]
    if out is None:
        if dev:
            raise ValueError("device evaluations need a preallocated out")
        out = np.empty((nrhs, npts))
    st = lib().hps_interpolate(h.ptr, _ptr(u), nrhs, _ptr(xy), npts, _ptr(out), 1 if dev else 0)
    if st != HPS_OK and check:
        raise HpsError(st, "hps_interpolate")
    return out if check else (out, st)


def hps_solve_static(h: Handle, f, u, check=True):
    """Solve through the allocation-free entry point (FP64 handle, device f and u)."""
    nrhs = 1 if f.ndim == 1 else f.shape[0]
    st = lib().hps_solve_static(h.ptr, _ptr(f), nrhs, _ptr(u))
    if st != HPS_OK and check:
        raise HpsError(st, "hps_solve_static")
    return st


def hps_query(h: Handle):
    nl, p, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb, by = ctypes.c_int64(), ctypes.c_int64()
    st = lib().hps_query(h.ptr, ctypes.byref(nl), ctypes.byref(p), ctypes.byref(q),
                         ctypes.byref(nb), ctypes.byref(by))
    if st != HPS_OK:
        raise HpsError(st, "hps_query")
    return {"n_leaves": nl.value, "p": p.value, "q": q.value, "nbnd": nb.value,
            "device_bytes": by.value}


def hps_free(h: Handle):
    h.close()


def hps_kernel_launches():
    return int(lib().hps_kernel_launches())


def hps_profile_enable(on=True):
    lib().hps_profile_enable(1 if on else 0)


def hps_profile_reset():
    lib().hps_profile_reset()


def hps_profile_read(max_out=64):
    """Per-kernel launch statistics since the last reset (synchronises the device)."""
    arr = (KernelStat * max_out)()
    n = lib().hps_profile_read(arr, max_out)
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms,
                                   "flops": arr[i].flops, "bytes": arr[i].bytes}
            for i in range(min(n, max_out))}


def _problem_struct(pr):
    P = Problem()
    P.d = _domain(pr["domain"])
    P.nx, P.ny, P.p, P.q = pr["nx"], pr["ny"], pr["p"], pr["q"]
    for k in COEFF_NAMES:
        setattr(P, k, _ptr(pr.get("coeffs", {}).get(k)))
    return P


def hps_estimate_bytes(problems, nrhs=1, precision=HPS_FP64, **kw):
    """(build_peak, resident, solve_workspace) in bytes for a list of problem dicts."""
    opt = _options(precision, False, None, kw.get("refine_tol"), kw.get("max_refine"),
                   kw.get("fp64_top_levels"), kw.get("form_root_dtn", False), kw.get("refine_depth"),
                   kw.get("leaf_refine"))
    arr = (Problem * len(problems))(*[_problem_struct(pr) for pr in problems])
    out = [ctypes.c_int64() for _ in range(3)]
    st = lib().hps_estimate_bytes(arr, len(problems), ctypes.byref(opt), nrhs,
                                  *[ctypes.byref(x) for x in out])
    if st != HPS_OK:
        raise HpsError(st, "hps_estimate_bytes")
    return tuple(x.value for x in out)


class Server:
    """The request loop of include/hps_serve.h."""

    def __init__(self, hbm_budget=0, workers=4, max_rhs_per_solve=256, device=0):
        o = ServerOptions()
        lib().hps_server_default_options(ctypes.byref(o))
        o.hbm_budget, o.workers, o.max_rhs_per_solve, o.device = (hbm_budget, workers,
                                                                  max_rhs_per_solve, device)
        out = ctypes.c_void_p()
        st = lib().hps_server_create(ctypes.byref(o), ctypes.byref(out))
        if st != HPS_OK:
            raise HpsError(st, "hps_server_create")
        self.ptr = out.value
        self.shapes = {}  # operator id -> (nl, p, nbnd)

    def submit_build(self, pr, precision=HPS_FP64, **kw):
        """pr: dict with domain, nx, ny, p, q and host coefficient arrays in 'coeffs'."""
        opt = _options(precision, False, None, kw.get("refine_tol"), kw.get("max_refine"),
                       kw.get("fp64_top_levels"), False, kw.get("refine_depth"),
                       kw.get("leaf_refine"))
        P = _problem_struct(pr)
        rid = lib().hps_server_submit_build(self.ptr, ctypes.byref(P), ctypes.byref(opt))
        if rid < 0:
            raise HpsError(int(rid), "hps_server_submit_build")
        self.shapes[rid] = (pr["nx"] * pr["ny"], pr["p"], hps_boundary_count(pr["nx"], pr["ny"], pr["q"]))
        return rid

    def submit_solve(self, op, f):
        f = np.ascontiguousarray(np.atleast_2d(f), dtype=np.float64)
        rid = lib().hps_server_submit_solve(self.ptr, op, f.ctypes.data, f.shape[0])
        if rid < 0:
            raise HpsError(int(rid), "hps_server_submit_solve")
        return rid

    def wait(self, rid, timeout=-1.0):
        info = RequestInfo()
        lib().hps_server_wait(self.ptr, rid, timeout, ctypes.byref(info))
        return info

    def result(self, rid, op, nrhs):
        nl, p, _ = self.shapes[op]
        u = np.empty((nrhs, nl, p, p))
        st = lib().hps_server_result(self.ptr, rid, u.ctypes.data)
        if st != HPS_OK:
            raise HpsError(st, "hps_server_result")
        return u

    def release(self, rid):
        return lib().hps_server_release(self.ptr, rid)

    def release_operator(self, op):
        return lib().hps_server_release_operator(self.ptr, op)

    def stats(self):
        s = ServerStats()
        lib().hps_server_get_stats(self.ptr, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}

    def close(self):
        if self.ptr:
            lib().hps_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
