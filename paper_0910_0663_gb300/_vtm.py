"""ctypes binding of libvtm (argument marshalling only).

Every function here has the name of the C entry point it calls (see
``include/vtm.h``) and does nothing but convert arguments: arrays may be
torch tensors (CPU or CUDA) or numpy arrays; their data pointers are passed
through unchanged.  Every step of the method runs inside libvtm.  If the
library is missing the import of this module fails loudly; there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvtm.so")

VTM_OK, VTM_EINVAL, VTM_ENOMEM, VTM_ESINGULAR, VTM_ENOCONV = 0, -1, -2, -3, -4
VTM_EDIVERGED, VTM_ETIMEOUT, VTM_ECUDA, VTM_EINTERNAL, VTM_ENOTFACTORED = -5, -6, -7, -8, -9
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
METHOD = {"vtm": 0, "bj": 1, "async": 2}
ADMITTANCE = {"alpha": 0, "diag": 1, "wob": 2, "sca": 3, "line": 4}


class vtm_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("check_every", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("method", ctypes.c_int), ("batch", ctypes.c_int),
                ("batch_solve", ctypes.c_int),
                ("l2_persist", ctypes.c_int), ("sweep_kernel", ctypes.c_int), ("graphs", ctypes.c_int),
                ("pdl", ctypes.c_int),
                ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_len", ctypes.c_int), ("batch_kernel", ctypes.c_int),
                ("wait_polls", ctypes.c_int), ("flow_lag", ctypes.c_int), ("band_solve", ctypes.c_int)]


class vtm_info(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("outer_steps", ctypes.c_int),
                ("relres", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("first_sweep_converged", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("sweep_launches", ctypes.c_int), ("t_sweeps_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vtm_plan_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nparts", ctypes.c_int32), ("nports", ctypes.c_int64),
                ("nlagged", ctypes.c_int64), ("sum_p2", ctypes.c_int64),
                ("max_ports", ctypes.c_int32), ("max_nodes", ctypes.c_int32),
                ("max_band", ctypes.c_int32), ("symmetric", ctypes.c_int32),
                ("t_bytes", ctypes.c_int64), ("factor_bytes", ctypes.c_int64),
                ("sweep_kernel", ctypes.c_int32), ("sum_tri", ctypes.c_int64),
                ("packed_bytes", ctypes.c_int64), ("batch_kernel", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VTMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.vtm_strerror(status).decode()
        detail = _lib.vtm_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({status}) {detail}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvtm.so not found at {LIB_PATH}: build it with "
                          "paper_0910_0663_gb300.build.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "vtm_plan": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, ctypes.POINTER(vtm_opts), P,
                                    ctypes.POINTER(P)]),
        "vtm_set_values": (ctypes.c_int, [P, P]),
        "vtm_set_opts": (ctypes.c_int, [P, ctypes.POINTER(vtm_opts)]),
        "vtm_set_admittance": (ctypes.c_int, [P, ctypes.c_int, dbl, ctypes.c_int, P]),
        "vtm_get_admittance": (ctypes.c_int, [P, P]),
        "vtm_factor": (ctypes.c_int, [P]),
        "vtm_solve": (ctypes.c_int, [P, P, P, i64, dbl, ctypes.POINTER(vtm_info)]),
        "vtm_adjoint": (ctypes.c_int, [P, P, P, i64, dbl, ctypes.POINTER(vtm_info)]),
        "vtm_march": (ctypes.c_int, [P, P, P, P, P, i64, dbl, ctypes.POINTER(vtm_info)]),
        "vtm_plan_get_stats": (ctypes.c_int, [P, ctypes.POINTER(vtm_plan_stats)]),
        "vtm_get_ports": (ctypes.c_int, [P, P, P, P, P]),
        "vtm_get_reflection": (ctypes.c_int, [P, i32, P, i64, ctypes.POINTER(i32)]),
        "vtm_get_reflection_stored": (ctypes.c_int, [P, i32, P, i64, ctypes.POINTER(i32),
                                                     ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "vtm_residual_norm": (ctypes.c_int, [P, P, P, i64, P]),
        "vtm_residual_norm_noalloc": (ctypes.c_int, [i64, P, P, P, P, P, i64, P, P]),
        "vtm_netmap_create": (ctypes.c_int, [i64, P, P, i64, P, P, P, ctypes.POINTER(P)]),
        "vtm_netmap_values": (ctypes.c_int, [P, P, P, P, P]),
        "vtm_netmap_gradient": (ctypes.c_int, [P, P, P, i64, P, P]),
        "vtm_netmap_destroy": (None, [P]),
        "vtm_destroy": (None, [P]),
        "vtm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "vtm_last_error_detail": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("vtm_plan", "vtm_set_values", "vtm_set_opts", "vtm_set_admittance",
            "vtm_get_admittance", "vtm_factor", "vtm_solve", "vtm_march",
            "vtm_adjoint", "vtm_plan_get_stats", "vtm_get_ports", "vtm_get_reflection",
            "vtm_get_reflection_stored",
            "vtm_residual_norm", "vtm_residual_norm_noalloc", "vtm_netmap_create",
            "vtm_netmap_values", "vtm_netmap_gradient", "vtm_netmap_destroy", "vtm_destroy",
            "vtm_strerror", "vtm_last_error_detail")


def _ptr(a):
    """Data pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(status, where):
    if status != VTM_OK:
        raise VTMError(status, where)


def make_opts(precision="fp64", max_sweeps=0, check_every=0, inner_tol=0.0, max_outer=0,
              history=None, sweep_kernel=0, method="vtm", batch=0, l2_persist=0, graphs=0,
              batch_solve=0, pdl=0, batch_kernel=0, wait_polls=0, flow_lag=0, band_solve=0):
    o = vtm_opts()
    o.band_solve = int(band_solve)
    o.batch_kernel = int(batch_kernel)
    o.wait_polls = int(wait_polls)
    o.flow_lag = int(flow_lag)
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.max_sweeps = max_sweeps
    o.check_every = check_every
    o.inner_tol = inner_tol
    o.max_outer = max_outer
    o.sweep_kernel = sweep_kernel
    o.method = METHOD[method] if isinstance(method, str) else int(method)
    o.batch = int(batch)
    o.l2_persist = int(l2_persist)
    o.graphs = int(graphs)
    o.pdl = int(pdl)
    o.batch_solve = int(batch_solve)
    if history is not None:
        assert history.dtype == np.float64 and history.flags["C_CONTIGUOUS"]
        o.history = history.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.history_len = int(history.size)
    return o


def vtm_plan(n, rowptr, colidx, vals, partition, nparts, Zc, opts=None, stream=0):
    h = ctypes.c_void_p()
    st = _lib.vtm_plan(int(n), _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(partition),
                       int(nparts), float(Zc), ctypes.byref(opts) if opts is not None else None,
                       ctypes.c_void_p(stream), ctypes.byref(h))
    _check(st, "vtm_plan")
    return h


def vtm_set_values(plan, vals):
    _check(_lib.vtm_set_values(plan, _ptr(vals)), "vtm_set_values")


def vtm_set_opts(plan, opts):
    _check(_lib.vtm_set_opts(plan, ctypes.byref(opts)), "vtm_set_opts")


def vtm_set_admittance(plan, kind, alpha=1.0, radius=2, W=None):
    k = ADMITTANCE[kind] if isinstance(kind, str) else int(kind)
    _check(_lib.vtm_set_admittance(plan, k, float(alpha), int(radius), _ptr(W)), "vtm_set_admittance")


def vtm_get_admittance(plan):
    W = np.empty(vtm_plan_get_stats(plan).nports, np.float64)
    _check(_lib.vtm_get_admittance(plan, _ptr(W)), "vtm_get_admittance")
    return W


def vtm_factor(plan):
    _check(_lib.vtm_factor(plan), "vtm_factor")


def vtm_solve(plan, b, x, nrhs, tol, check=True):
    info = vtm_info()
    st = _lib.vtm_solve(plan, _ptr(b), _ptr(x), int(nrhs), float(tol), ctypes.byref(info))
    if check:
        _check(st, "vtm_solve")
    return st, info


def vtm_adjoint(plan, g, lam, nrhs, tol, check=True):
    info = vtm_info()
    st = _lib.vtm_adjoint(plan, _ptr(g), _ptr(lam), int(nrhs), float(tol), ctypes.byref(info))
    if check:
        _check(st, "vtm_adjoint")
    return st, info


def vtm_march(plan, cdiag, p, x0, X, nsteps, tol, check=True):
    info = vtm_info()
    st = _lib.vtm_march(plan, _ptr(cdiag), _ptr(p), _ptr(x0), _ptr(X), int(nsteps), float(tol),
                        ctypes.byref(info))
    if check:
        _check(st, "vtm_march")
    return st, info


def vtm_plan_get_stats(plan):
    s = vtm_plan_stats()
    _check(_lib.vtm_plan_get_stats(plan, ctypes.byref(s)), "vtm_plan_get_stats")
    return s


def vtm_get_ports(plan):
    m = vtm_plan_get_stats(plan).nports
    out = [np.empty(m, np.int32) for _ in range(4)]
    _check(_lib.vtm_get_ports(plan, *[_ptr(a) for a in out]), "vtm_get_ports")
    return tuple(out)


def vtm_get_reflection(plan, part):
    p = ctypes.c_int32()
    _check(_lib.vtm_get_reflection(plan, int(part), None, 0, ctypes.byref(p)), "vtm_get_reflection")
    T = np.empty((p.value, p.value), np.float64)
    _check(_lib.vtm_get_reflection(plan, int(part), _ptr(T), T.size, ctypes.byref(p)),
           "vtm_get_reflection")
    return T


def vtm_get_reflection_stored(plan, part):
    """(T, element bytes, packed) -- T_P as the plan's sweeps read it, in FP64."""
    p, es, pk = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.vtm_get_reflection_stored(plan, int(part), None, 0, ctypes.byref(p), ctypes.byref(es),
                                          ctypes.byref(pk)), "vtm_get_reflection_stored")
    T = np.empty((p.value, p.value), np.float64)
    _check(_lib.vtm_get_reflection_stored(plan, int(part), _ptr(T), T.size, ctypes.byref(p), ctypes.byref(es),
                                          ctypes.byref(pk)), "vtm_get_reflection_stored")
    return T, es.value, bool(pk.value)


def vtm_residual_norm(plan, x, b, nrhs):
    rel = np.empty(int(nrhs), np.float64)
    _check(_lib.vtm_residual_norm(plan, _ptr(x), _ptr(b), int(nrhs), _ptr(rel)), "vtm_residual_norm")
    return rel


def vtm_destroy(plan):
    _lib.vtm_destroy(plan)


def vtm_strerror(status):
    return _lib.vtm_strerror(int(status)).decode()


def vtm_last_error_detail():
    return _lib.vtm_last_error_detail().decode()


def vtm_residual_norm_noalloc(n, rowptr, colidx, vals, x, b, nrhs, stream=0):
    """Relative residual norms with no plan and no device allocation (all
    arrays on the device; see include/vtm.h)."""
    rel = np.empty(int(nrhs), np.float64)
    _check(_lib.vtm_residual_norm_noalloc(int(n), _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(x),
                                          _ptr(b), int(nrhs), _ptr(rel), ctypes.c_void_p(stream)),
           "vtm_residual_norm_noalloc")
    return rel


def vtm_netmap_create(n, rowptr, colidx, nedges, ei, ej, stream=0):
    h = ctypes.c_void_p()
    _check(_lib.vtm_netmap_create(int(n), _ptr(rowptr), _ptr(colidx), int(nedges), _ptr(ei), _ptr(ej),
                                  ctypes.c_void_p(stream), ctypes.byref(h)), "vtm_netmap_create")
    return h


def vtm_netmap_values(netmap, rowptr, g, ground, vals):
    _check(_lib.vtm_netmap_values(netmap, _ptr(rowptr), _ptr(g), _ptr(ground), _ptr(vals)),
           "vtm_netmap_values")


def vtm_netmap_gradient(netmap, lam, x, nrhs, grad_g, grad_ground=None):
    _check(_lib.vtm_netmap_gradient(netmap, _ptr(lam), _ptr(x), int(nrhs), _ptr(grad_g),
                                    _ptr(grad_ground)), "vtm_netmap_gradient")


def vtm_netmap_destroy(netmap):
    _lib.vtm_netmap_destroy(netmap)
