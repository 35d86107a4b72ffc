"""CPU FP64 oracle for HPR-QP: TEST INFRASTRUCTURE ONLY.

The plain C oracle (``hprqp_oracle.c``) implements Algorithm 4 of arXiv 2507.02470 step by
step; this module compiles it with gcc and marshals ``qpgen.QP`` objects into its structs.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libhprqp_oracle.so")
_lock = threading.Lock()
_lib = None

QKIND = {"diag": 1, "csr": 2, "dia": 3, "factor": 4, "dense_factor": 5, "qap": 6}
STATUS = {0: "converged", 1: "max_iter", 3: "numerical_error", 4: "invalid_arg"}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no fused multiply-add)."""
    src = os.path.join(_HERE, "hprqp_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "hprqp_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _QTerm(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_int64), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("vals", C.c_void_p), ("ndiag", C.c_int32), ("offsets", C.c_void_p), ("diags", C.c_void_p),
                ("dense", C.c_void_p)]


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("nq", C.c_int32), ("q", C.POINTER(_QTerm)),
                ("A_rowptr", C.c_void_p), ("A_colidx", C.c_void_p), ("A_vals", C.c_void_p),
                ("c", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p), ("L", C.c_void_p),
                ("U", C.c_void_p), ("phi", C.c_int32), ("lam", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("check_every", C.c_int64),
                ("restart_every", C.c_int64), ("alpha1", C.c_double), ("alpha2", C.c_double),
                ("alpha3", C.c_double), ("alpha3_tight", C.c_double), ("ratio_tight", C.c_double),
                ("lambda_A", C.c_double), ("lambda_Q", C.c_double), ("sigma0", C.c_double),
                ("power_max_iter", C.c_int64), ("power_tol", C.c_double), ("power_safety", C.c_double),
                ("halpern_total", C.c_int32), ("sigma_golden", C.c_int32), ("restart_off", C.c_int32),
                ("sigma_fixed", C.c_int32), ("scaling", C.c_int32), ("method", C.c_int32), ("x0", C.c_void_p), ("y0", C.c_void_p),
                ("trace_len", C.c_int64), ("trace_x", C.c_void_p), ("trace_y", C.c_void_p),
                ("trace_R", C.c_void_p), ("trace_sigma", C.c_void_p), ("trace_restart", C.c_void_p),
                ("trace_w", C.c_void_p)]


class _Result(C.Structure):
    _fields_ = [("eta_p", C.c_double), ("eta_d", C.c_double), ("eta_gap", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("iters", C.c_int64),
                ("restarts", C.c_int64), ("sigma", C.c_double), ("lambda_A", C.c_double),
                ("lambda_Q", C.c_double), ("status", C.c_int32), ("iters_1e4", C.c_int64),
                ("iters_1e6", C.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, dbl, i64 = C.c_void_p, C.c_double, C.c_int64
            L.orc_default_params.argtypes = [C.POINTER(_Params)]
            L.orc_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_Result), vp, vp, vp, vp]
            L.orc_solve.restype = C.c_int
            L.orc_scaling.argtypes = [C.POINTER(_Problem), vp, vp]
            L.orc_scaling.restype = C.c_int
            for f in (L.orc_qmul, L.orc_amul, L.orc_atmul):
                f.argtypes = [C.POINTER(_Problem), vp, vp]
            for f in (L.orc_power_A, L.orc_power_Q):
                f.argtypes = [C.POINTER(_Problem), i64, dbl, dbl]
                f.restype = dbl
            L.orc_sigma_argmin.argtypes = [dbl, dbl, dbl, dbl, C.c_int]
            L.orc_sigma_argmin.restype = dbl
            L.orc_sigma_update.argtypes = [dbl, dbl, dbl, dbl, dbl, dbl, C.c_int]
            L.orc_sigma_update.restype = dbl
            L.orc_mnorm2.argtypes = [C.POINTER(_Problem), dbl, dbl, dbl, vp, vp, vp]
            L.orc_mnorm2.restype = dbl
            L.orc_eta.argtypes = [C.POINTER(_Problem), vp, vp, vp, vp, vp, vp]
            L.orc_step.argtypes = [C.POINTER(_Problem), dbl, dbl, dbl, vp, vp, vp, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class Problem:
    """Keeps the numpy buffers alive for as long as the C struct refers to them."""

    def __init__(self, qp):
        self.qp = qp
        self._keep = []
        f64 = lambda a: self._hold(np.ascontiguousarray(a, dtype=np.float64))
        i32 = lambda a: self._hold(np.ascontiguousarray(a, dtype=np.int32))
        terms = (_QTerm * max(1, len(qp.qterms)))()
        for k, t in enumerate(qp.qterms):
            tt = terms[k]
            tt.kind = QKIND[t.kind]
            tt.p = int(t.p)
            if t.rowptr is not None:
                tt.rowptr = _ptr(i32(t.rowptr))
                tt.colidx = _ptr(i32(t.colidx))
                tt.vals = _ptr(f64(t.vals))
            if t.offsets is not None:
                tt.ndiag = len(t.offsets)
                tt.offsets = _ptr(i32(t.offsets))
                tt.diags = _ptr(f64(np.asarray(t.diags).reshape(-1)))
            if t.dense is not None:
                tt.dense = _ptr(f64(np.asarray(t.dense).reshape(-1)))
        self._terms = terms
        s = _Problem()
        s.n, s.m, s.nq = qp.n, qp.m, len(qp.qterms)
        s.q = C.cast(terms, C.POINTER(_QTerm))
        s.A_rowptr = _ptr(i32(qp.A_rowptr))
        s.A_colidx = _ptr(i32(qp.A_colidx if qp.A_colidx.size else np.zeros(1, np.int32)))
        s.A_vals = _ptr(f64(qp.A_vals if qp.A_vals.size else np.zeros(1)))
        s.c = _ptr(f64(qp.c))
        s.l = _ptr(f64(qp.l if qp.m else np.zeros(1)))
        s.u = _ptr(f64(qp.u if qp.m else np.zeros(1)))
        s.L = _ptr(f64(qp.L))
        s.U = _ptr(f64(qp.U))
        s.phi = qp.phi
        s.lam = float(qp.lam)
        self.s = s

    def _hold(self, a):
        self._keep.append(a)
        return a

    @property
    def ref(self):
        return C.byref(self.s)


@dataclass
class Solution:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    w: np.ndarray
    eta_p: float
    eta_d: float
    eta_gap: float
    pobj: float
    dobj: float
    iters: int
    restarts: int
    sigma: float
    lambda_A: float
    lambda_Q: float
    status: str
    trace: Optional[dict] = None
    iters_1e4: int = 0
    iters_1e6: int = 0


def default_params() -> dict:
    p = _Params()
    lib().orc_default_params(C.byref(p))
    return {name: getattr(p, name) for name, _ in _Params._fields_
            if not name.startswith("trace") and name not in ("x0", "y0")}


def solve(qp, trace_len: int = 0, x0=None, y0=None, **kw) -> Solution:
    """Run Algorithm 4 on ``qp``; keyword arguments override the Sec. 4.1 defaults."""
    L = lib()
    P = Problem(qp)
    p = _Params()
    L.orc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    keep = []
    if x0 is not None:
        x0 = np.ascontiguousarray(x0, np.float64); keep.append(x0); p.x0 = x0.ctypes.data
    if y0 is not None:
        y0 = np.ascontiguousarray(y0, np.float64); keep.append(y0); p.y0 = y0.ctypes.data
    tr = None
    if trace_len > 0:
        tr = {"x": np.zeros((trace_len, qp.n)), "y": np.zeros((trace_len, max(qp.m, 1))),
              "w": np.zeros((trace_len, qp.n)),
              "R": np.full(trace_len, np.nan), "sigma": np.zeros(trace_len),
              "restart": np.zeros(trace_len, np.int32)}
        p.trace_len = trace_len
        p.trace_x = tr["x"].ctypes.data
        p.trace_y = tr["y"].ctypes.data
        p.trace_R = tr["R"].ctypes.data
        p.trace_sigma = tr["sigma"].ctypes.data
        p.trace_restart = tr["restart"].ctypes.data
        p.trace_w = tr["w"].ctypes.data
    r = _Result()
    x = np.zeros(qp.n); y = np.zeros(max(qp.m, 1)); z = np.zeros(qp.n); w = np.zeros(qp.n)
    L.orc_solve(P.ref, C.byref(p), C.byref(r), x.ctypes.data, y.ctypes.data, z.ctypes.data, w.ctypes.data)
    if tr is not None:
        it = int(min(r.iters, trace_len))
        tr = {k: v[:it] for k, v in tr.items()}
        if qp.m == 0:
            tr["y"] = tr["y"][:, :0]
    return Solution(x, y[:qp.m], z, w, r.eta_p, r.eta_d, r.eta_gap, r.pobj, r.dobj, int(r.iters),
                    int(r.restarts), r.sigma, r.lambda_A, r.lambda_Q, STATUS.get(r.status, str(r.status)), tr,
                    int(r.iters_1e4), int(r.iters_1e6))


def scaling(qp):
    """(d, e, applied): the Sec. 4.1 preconditioning of qp (x = D xs, y = E ys)."""
    P = Problem(qp)
    d = np.ones(qp.n)
    e = np.ones(max(qp.m, 1))
    ok = lib().orc_scaling(P.ref, d.ctypes.data, e.ctypes.data)
    return d, e[:qp.m], bool(ok)


def qmul(qp, v):
    P = Problem(qp); v = np.ascontiguousarray(v, np.float64); out = np.zeros(qp.n)
    lib().orc_qmul(P.ref, v.ctypes.data, out.ctypes.data); return out


def amul(qp, v):
    P = Problem(qp); v = np.ascontiguousarray(v, np.float64); out = np.zeros(max(qp.m, 1))
    lib().orc_amul(P.ref, v.ctypes.data, out.ctypes.data); return out[:qp.m]


def atmul(qp, v):
    P = Problem(qp); v = np.ascontiguousarray(v, np.float64); out = np.zeros(qp.n)
    lib().orc_atmul(P.ref, v.ctypes.data if v.size else None, out.ctypes.data); return out


def power_A(qp, max_iter=5000, tol=1e-6, safety=1.01):
    return lib().orc_power_A(Problem(qp).ref, max_iter, tol, safety)


def power_Q(qp, max_iter=5000, tol=1e-6, safety=1.01):
    return lib().orc_power_Q(Problem(qp).ref, max_iter, tol, safety)


def sigma_argmin(t1, t2, t3, lamQ, golden=False):
    return lib().orc_sigma_argmin(t1, t2, t3, lamQ, int(golden))


def sigma_update(t1, t2, t3, lamQ, ratio, sigma_r, golden=False):
    return lib().orc_sigma_update(t1, t2, t3, lamQ, ratio, sigma_r, int(golden))


def mnorm2(qp, sigma, lamA, lamQ, dy, dw, dx):
    P = Problem(qp)
    dy = np.ascontiguousarray(dy, np.float64) if qp.m else np.zeros(1)
    dw = np.ascontiguousarray(dw, np.float64); dx = np.ascontiguousarray(dx, np.float64)
    return lib().orc_mnorm2(P.ref, sigma, lamA, lamQ, dy.ctypes.data, dw.ctypes.data, dx.ctypes.data)


def eta(qp, xb, yb, zb):
    P = Problem(qp)
    xb = np.ascontiguousarray(xb, np.float64); zb = np.ascontiguousarray(zb, np.float64)
    yb = np.ascontiguousarray(yb, np.float64) if qp.m else np.zeros(1)
    e = np.zeros(3); po = C.c_double(); do = C.c_double()
    lib().orc_eta(P.ref, xb.ctypes.data, yb.ctypes.data, zb.ctypes.data, e.ctypes.data,
                  C.addressof(po), C.addressof(do))
    return e, po.value, do.value


def step(qp, sigma, lamA, lamQ, y, w, x):
    """One fixed-sigma inner step of Algorithm 3; returns (yb, wb, zb, xb, wh)."""
    P = Problem(qp)
    n, m = qp.n, qp.m
    y = np.ascontiguousarray(y, np.float64) if m else np.zeros(1)
    w = np.ascontiguousarray(w, np.float64); x = np.ascontiguousarray(x, np.float64)
    yb = np.zeros(max(m, 1)); wb = np.zeros(n); zb = np.zeros(n); xb = np.zeros(n); wh = np.zeros(n)
    lib().orc_step(P.ref, sigma, lamA, lamQ, y.ctypes.data, w.ctypes.data, x.ctypes.data,
                   yb.ctypes.data, wb.ctypes.data, zb.ctypes.data, xb.ctypes.data, wh.ctypes.data)
    return yb[:m], wb, zb, xb, wh
