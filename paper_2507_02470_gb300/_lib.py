"""ctypes binding of the C ABI in include/hprqp.h (argument marshalling only).

Every computation runs inside libhprqp.so on the GPU.  The library must be built first
(``paper_2507_02470_gb300.build.build()``); loading raises if it is missing.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB as _LIB_PATH

_lock = threading.Lock()
_lib = None

HPRQP_OK, HPRQP_MAX_ITER, HPRQP_TIME_LIMIT, HPRQP_NUMERICAL_ERROR = 0, 1, 2, 3
HPRQP_INVALID_ARG, HPRQP_CUDA_ERROR, HPRQP_TIMEOUT, HPRQP_OOM = 4, 5, 6, 7
STATUS_NAMES = {0: "converged", 1: "max_iter", 2: "time_limit", 3: "numerical_error", 4: "invalid_arg",
                5: "cuda_error", 6: "timeout", 7: "oom"}
QKIND = {"diag": 1, "csr": 2, "dia": 3, "factor": 4, "dense_factor": 5, "qap": 6}

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class hprqp_qterm(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("colidx", C.c_void_p), ("vals", C.c_void_p), ("ndiag", C.c_int32), ("offsets", C.c_void_p),
                ("diags", C.c_void_p), ("dense", C.c_void_p)]


class hprqp_qop(C.Structure):
    _fields_ = [("nterms", C.c_int32), ("terms", C.POINTER(hprqp_qterm))]


class hprqp_params(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("check_every", C.c_int64), ("restart_every", C.c_int64),
                ("alpha1", C.c_double), ("alpha2", C.c_double), ("alpha3", C.c_double),
                ("alpha3_tight", C.c_double), ("ratio_tight", C.c_double), ("lambda_A", C.c_double),
                ("lambda_Q", C.c_double), ("sigma0", C.c_double), ("power_max_iter", C.c_int64),
                ("power_tol", C.c_double), ("power_safety", C.c_double), ("halpern_total", C.c_int32),
                ("sigma_golden", C.c_int32), ("restart_off", C.c_int32), ("sigma_fixed", C.c_int32),
                ("time_limit", C.c_double), ("iters_per_launch", C.c_int32), ("autotune", C.c_int32),
                ("verbose", C.c_int32), ("alloc", _ALLOC_FN), ("free", _FREE_FN), ("alloc_ctx", C.c_void_p),
                ("launch_mode", C.c_int32), ("scaling", C.c_int32), ("method", C.c_int32),
                ("pdl", C.c_int32), ("fixed_schedule", C.c_int32),
                ("tiled_factor", C.c_int32), ("fused_steps", C.c_int32), ("factor_inline", C.c_int32),
                ("wait_polls", C.c_int32), ("batch_team", C.c_int32)]


class hprqp_kkt(C.Structure):
    _fields_ = [("eta_p", C.c_double), ("eta_d", C.c_double), ("eta_gap", C.c_double), ("rel_kkt", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("iters", C.c_int64), ("restarts", C.c_int64),
                ("sigma", C.c_double), ("lambda_A", C.c_double), ("lambda_Q", C.c_double),
                ("solve_seconds", C.c_double), ("power_seconds", C.c_double), ("kernel_launches", C.c_int64),
                ("status", C.c_int32), ("iters_1e4", C.c_int64), ("iters_1e6", C.c_int64),
                ("seconds_1e4", C.c_double), ("seconds_1e6", C.c_double), ("lanes_q", C.c_int32),
                ("lanes_a", C.c_int32), ("lanes_at", C.c_int32), ("lanes_pre", C.c_int32),
                ("tiled_terms", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status"] = STATUS_NAMES.get(d["status"], str(d["status"]))
        return d


class hprqp_check(C.Structure):
    _fields_ = [("iter", C.c_int64), ("restarts", C.c_int64), ("sigma", C.c_double), ("eta_p", C.c_double),
                ("eta_d", C.c_double), ("eta_gap", C.c_double), ("pobj", C.c_double), ("dobj", C.c_double),
                ("R", C.c_double), ("seconds", C.c_double)]


class hprqp_problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("Q", C.POINTER(hprqp_qop)), ("A_rowptr", C.c_void_p),
                ("A_colidx", C.c_void_p), ("A_vals", C.c_void_p), ("c", C.c_void_p), ("l", C.c_void_p),
                ("u", C.c_void_p), ("L", C.c_void_p), ("U", C.c_void_p), ("phi", C.c_int32), ("lam", C.c_double),
                ("x0", C.c_void_p), ("y0", C.c_void_p), ("sigma0", C.c_double), ("lambda_A", C.c_double),
                ("lambda_Q", C.c_double)]


# (name, restype, argtypes) of every exported symbol declared in include/hprqp.h
_vp, _i32, _i64, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
SIGNATURES = [
    ("hprqp_default_params", None, [C.POINTER(hprqp_params)]),
    ("hprqp_create", C.c_int, [C.POINTER(_vp), _i64, _i64, C.POINTER(hprqp_qop), _vp, _vp, _vp, _vp, _vp, _vp,
                               _vp, _vp, _i32, _dbl, C.POINTER(hprqp_params)]),
    ("hprqp_set_warm_start", C.c_int, [_vp, _vp, _vp, _dbl]),
    ("hprqp_solve", C.c_int, [_vp, _dbl, _i64]),
    ("hprqp_get", C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(hprqp_kkt)]),
    ("hprqp_apply", C.c_int, [_vp, _i32, _vp, _vp]),
    ("hprqp_profile", C.c_int, [_vp, _i32, _vp]),
    ("hprqp_power_noalloc", C.c_int, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _dbl, _dbl, _vp,
                                      C.POINTER(_dbl)]),
    ("hprqp_destroy", None, [_vp]),
    ("hprqp_batch_create", C.c_int, [C.POINTER(_vp), _i32, C.POINTER(hprqp_problem), C.POINTER(hprqp_params)]),
    ("hprqp_batch_solve", C.c_int, [_vp, _dbl, _i64]),
    ("hprqp_batch_get", C.c_int, [_vp, _i32, _vp, _vp, _vp, C.POINTER(hprqp_kkt)]),
    ("hprqp_batch_stats", C.c_int, [_vp, C.POINTER(_dbl), C.POINTER(_i64)]),
    ("hprqp_batch_schedule", C.c_int, [_vp, _vp]),
    ("hprqp_batch_destroy", None, [_vp]),
    ("hprqp_batch_last_error", C.c_char_p, [_vp]),
    ("hprqp_last_error", C.c_char_p, [_vp]),
    ("hprqp_set_data", C.c_int, [_vp, _vp, _vp, _vp]),
    ("hprqp_history", C.c_int, [_vp, _vp, _i32, C.POINTER(_i32)]),
    ("hprqp_set_lambda", C.c_int, [_vp, _dbl, _dbl]),
    ("hprqp_fp64_rate", C.c_int, [_i32, _i32, C.POINTER(_dbl), C.POINTER(_dbl), C.POINTER(_dbl)]),
    ("hprqp_memory_stats", C.c_int, [_vp, _vp]),
    ("hprqp_set_wait_polls", C.c_int, [_vp, _i32]),
    # learned warm start (include/hprqp_learn.h)
    ("hprqp_gemm_bf16", C.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp]),
    ("hprqp_learn_check", C.c_int, []),
    ("hprqp_cast_bf16_f64", C.c_int, [_vp, _i64, _i64, _i64, _vp, _dbl, _vp, _i64, _vp, _vp]),
    ("hprqp_cast_bf16_f32", C.c_int, [_vp, _i64, _i64, _i64, _vp, _dbl, _vp, _i64, _vp, _vp]),
    ("hprqp_row_stats", C.c_int, [_vp, _i64, _i64, _i64, C.c_float, _vp, _vp, _vp]),
    ("hprqp_col_mean_f64", C.c_int, [_vp, _i64, _i64, _i64, _vp, _vp]),
    ("hprqp_ws_standardize", C.c_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _i64, _vp]),
    ("hprqp_mlp_create", C.c_int, [C.POINTER(_vp), _i32, C.POINTER(_i32), _i32, _vp]),
    ("hprqp_mlp_set_layer", C.c_int, [_vp, _i32, _vp, _vp]),
    ("hprqp_mlp_get_layer", C.c_int, [_vp, _i32, _vp, _vp]),
    ("hprqp_mlp_forward", C.c_int, [_vp, _vp, _i64, _i32, _vp, _i64]),
    ("hprqp_mlp_backward", C.c_int, [_vp, _vp, _i64]),
    ("hprqp_mlp_get_grad", C.c_int, [_vp, _i32, _vp, _vp]),
    ("hprqp_mlp_adam", C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float, _i64]),
    ("hprqp_mlp_destroy", C.c_int, [_vp]),
    ("hprqp_ws_loss", C.c_int, [_vp, _i64, _i32, _i32, _vp, _vp, _i64, _vp, _vp, C.c_float, C.c_float, C.c_float,
                                C.c_float, C.c_float, _vp, _i64, _i32, _vp, _vp]),
    ("hprqp_ws_decode", C.c_int, [_vp, _i64, _i64, _i32, _vp, _i64, _i32, C.c_float, C.c_float, C.c_float, _vp, _vp,
                                  _vp, _vp, _vp, _i64, _vp, _vp]),
    ("hprqp_learn_last_error", C.c_char_p, []),
]


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libhprqp.so (raises OSError/RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} (run paper_2507_02470_gb300.build.build())")
            L = C.CDLL(path)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class HPRQPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (host or CUDA), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def default_params() -> hprqp_params:
    p = hprqp_params()
    lib().hprqp_default_params(C.byref(p))
    return p


def fp64_rate(op=0, lanes=32):
    """Issue rate of one arithmetic operation on the current device (hprqp_fp64_rate):
    op 0 FP64 FMA, 1 FP64 add, 2 FP64 multiply, 3 FP32 FMA.  Returns a dict with the thread
    operations per SM clock per SM, the SM clock (MHz) during the run and the device-wide
    thread operations per second."""
    r, mhz, ops = C.c_double(), C.c_double(), C.c_double()
    st = lib().hprqp_fp64_rate(int(op), int(lanes), C.byref(r), C.byref(mhz), C.byref(ops))
    if st != HPRQP_OK:
        raise HPRQPError(st, "hprqp_fp64_rate failed")
    return {"lanes_per_clk": r.value, "sm_mhz": mhz.value, "ops_per_s": ops.value}


def _torch_cuda() -> bool:
    try:
        import torch
        return bool(torch.cuda.is_available())
    except Exception:
        return False


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator (blocks
    tied to the handle's stream; the handle synchronizes that stream before it frees them)."""

    def __init__(self):
        import torch

        self.torch = torch
        self.count = 0

        def _alloc(nbytes, ctx, stream):
            try:
                p = self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
                self.count += 1
                return p
            except Exception:
                return None

        def _free(ptr, nbytes, ctx, stream):
            self.torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = _ALLOC_FN(_alloc)
        self.free = _FREE_FN(_free)


class Solver:
    """One HPR-QP instance on the GPU (a handle of the C ABI).

    ``qp`` is any object with the fields n, m, A_rowptr, A_colidx, A_vals, c, l, u, L, U,
    phi, lam and qterms (a list of terms with kind, p, rowptr, colidx, vals, offsets, diags,
    dense); arrays may be numpy (host) or torch CUDA tensors (device).
    """

    def __init__(self, qp, stream=None, torch_alloc=None, **params):
        L = lib()
        self._keep = []
        p = default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        if stream is not None:
            p.stream = int(stream)
        self._alloc = None
        # device memory through PyTorch's caching allocator unless the caller says otherwise
        # (torch_alloc=False: the library's own cudaMalloc path)
        if torch_alloc is None:
            torch_alloc = _torch_cuda()
        if torch_alloc:
            self._alloc = _TorchAllocator()
            p.alloc = self._alloc.alloc
            p.free = self._alloc.free
        self.params = p
        terms = (hprqp_qterm * max(1, len(qp.qterms)))()
        for k, t in enumerate(qp.qterms):
            tt = terms[k]
            tt.kind = QKIND[t.kind]
            tt.p = int(getattr(t, "p", 0) or 0)
            if t.rowptr is not None:
                rp, ci, va = self._hold(t.rowptr, np.int32), self._hold(t.colidx, np.int32), self._hold(t.vals, np.float64)
                tt.rowptr, tt.colidx, tt.vals = _ptr(rp), _ptr(ci), _ptr(va)
                tt.nnz = int(ci.shape[0])
            if t.offsets is not None:
                tt.ndiag = len(t.offsets)
                tt.offsets = _ptr(self._hold(t.offsets, np.int32))
                tt.diags = _ptr(self._hold(t.diags, np.float64))
            if t.dense is not None:
                tt.dense = _ptr(self._hold(t.dense, np.float64))
        qop = hprqp_qop(len(qp.qterms), C.cast(terms, C.POINTER(hprqp_qterm)))
        self.n, self.m = int(qp.n), int(qp.m)
        h = C.c_void_p()
        st = L.hprqp_create(C.byref(h), self.n, self.m, C.byref(qop),
                            _ptr(self._hold(qp.A_rowptr, np.int32)) if self.m else None,
                            _ptr(self._hold(qp.A_colidx, np.int32)) if self.m else None,
                            _ptr(self._hold(qp.A_vals, np.float64)) if self.m else None,
                            _ptr(self._hold(qp.c, np.float64)),
                            _ptr(self._hold(qp.l, np.float64)) if self.m else None,
                            _ptr(self._hold(qp.u, np.float64)) if self.m else None,
                            _ptr(self._hold(qp.L, np.float64)) if qp.L is not None else None,
                            _ptr(self._hold(qp.U, np.float64)) if qp.U is not None else None,
                            int(qp.phi), float(qp.lam), C.byref(p))
        self._keep = []  # inputs are copied by hprqp_create
        if st != HPRQP_OK:
            raise HPRQPError(st, L.hprqp_last_error(None).decode())
        self.h = h

    def _hold(self, a, dtype):
        if hasattr(a, "data_ptr"):
            import torch
            tdt = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
            a = a.to(tdt).contiguous()
        else:
            a = np.ascontiguousarray(a, dtype=dtype)
        self._keep.append(a)
        return a

    def _check(self, st, ok=(HPRQP_OK,)):
        if st not in ok:
            raise HPRQPError(st, lib().hprqp_last_error(self.h).decode())
        return st

    def set_warm_start(self, x0=None, y0=None, sigma0=0.0):
        keep = [None if x0 is None else self._hold(x0, np.float64),
                None if y0 is None else self._hold(y0, np.float64)]
        self._check(lib().hprqp_set_warm_start(self.h, _ptr(keep[0]), _ptr(keep[1]), float(sigma0)))
        self._keep = []

    def set_data(self, c=None, l=None, u=None):
        """Replaces c and the row bounds (host numpy or CUDA tensors; None keeps them)."""
        keep = [None if a is None else self._hold(a, np.float64) for a in (c, l, u)]
        self._check(lib().hprqp_set_data(self.h, *[_ptr(a) for a in keep]))
        self._keep = []

    def set_wait_polls(self, polls):
        """launch_mode 3: polls of one grid-barrier wait before the solve gives up (0: default)."""
        self._check(lib().hprqp_set_wait_polls(self.h, int(polls)))

    def set_lambda(self, lambda_A, lambda_Q):
        """Fixes lambda_A, lambda_Q for later solves (0 restores the power method)."""
        self._check(lib().hprqp_set_lambda(self.h, float(lambda_A), float(lambda_Q)))

    def solve(self, tol=1e-8, max_iter=1_000_000):
        st = lib().hprqp_solve(self.h, float(tol), int(max_iter))
        self._check(st, ok=(HPRQP_OK, HPRQP_MAX_ITER, HPRQP_TIME_LIMIT, HPRQP_NUMERICAL_ERROR))
        return STATUS_NAMES[st]

    def get(self, x=None, y=None, z=None, w=None):
        """Copies the bar iterate into the given buffers (numpy or torch; None = allocate
        numpy arrays) and returns (x, y, z, w, kkt dict)."""
        x = np.empty(self.n) if x is None else x
        y = np.empty(self.m) if y is None else y
        z = np.empty(self.n) if z is None else z
        w = np.empty(self.n) if w is None else w
        k = hprqp_kkt()
        self._check(lib().hprqp_get(self.h, _ptr(x), _ptr(y) if self.m else None, _ptr(z), _ptr(w), C.byref(k)))
        return x, y, z, w, k.as_dict()

    def kkt(self):
        k = hprqp_kkt()
        self._check(lib().hprqp_get(self.h, None, None, None, None, C.byref(k)))
        return k.as_dict()

    def memory_stats(self):
        """Device memory the handle holds, by path (hprqp_memory_stats)."""
        out = np.zeros(4, np.int64)
        self._check(lib().hprqp_memory_stats(self.h, _ptr(out)))
        return {"hook_allocs": int(out[0]), "hook_bytes": int(out[1]), "cudamalloc_allocs": int(out[2]),
                "cudamalloc_bytes": int(out[3])}

    def history(self, cap=512):
        """The stopping tests of the last solve (oldest first) as a list of dicts."""
        buf = (hprqp_check * cap)()
        cnt = _i32(0)
        self._check(lib().hprqp_history(self.h, C.cast(buf, _vp), cap, C.byref(cnt)))
        return [{k: getattr(buf[i], k) for k, _ in hprqp_check._fields_} for i in range(cnt.value)]

    def apply(self, op, v):
        """op 'A' (n -> m), 'AT' (m -> n) or 'Q' (n -> n) applied on the GPU."""
        code = {"A": 0, "AT": 1, "Q": 2}[op]
        v = np.ascontiguousarray(v, np.float64)
        out = np.empty(self.m if code == 0 else self.n)
        self._check(lib().hprqp_apply(self.h, code, _ptr(v), _ptr(out)))
        return out

    PROFILE_KINDS = ["zx", "pre1", "q1", "a1", "at", "pre2", "q2", "restart_pre", "restart", "ath", "prew", "q2h"]

    def profile(self, iters=20):
        """Mean per-kernel durations (ms) of `iters` inner steps, timed with CUDA events."""
        ms = np.zeros(len(self.PROFILE_KINDS))
        self._check(lib().hprqp_profile(self.h, int(iters), _ptr(ms)))
        return dict(zip(self.PROFILE_KINDS, ms.tolist()))

    def close(self):
        if getattr(self, "h", None):
            lib().hprqp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _qop_of(qp, hold):
    terms = (hprqp_qterm * max(1, len(qp.qterms)))()
    for k, t in enumerate(qp.qterms):
        tt = terms[k]
        tt.kind = QKIND[t.kind]
        tt.p = int(getattr(t, "p", 0) or 0)
        if t.rowptr is not None:
            rp, ci, va = hold(t.rowptr, np.int32), hold(t.colidx, np.int32), hold(t.vals, np.float64)
            tt.rowptr, tt.colidx, tt.vals = _ptr(rp), _ptr(ci), _ptr(va)
            tt.nnz = int(ci.shape[0])
        if t.offsets is not None:
            tt.ndiag = len(t.offsets)
            tt.offsets = _ptr(hold(t.offsets, np.int32))
            tt.diags = _ptr(hold(t.diags, np.float64))
        if t.dense is not None:
            tt.dense = _ptr(hold(t.dense, np.float64))
    hold(terms, None)
    q = hprqp_qop(len(qp.qterms), C.cast(terms, C.POINTER(hprqp_qterm)))
    hold(q, None)
    return q


class BatchSolver:
    """Many independent QPs solved in one persistent launch (hprqp_batch_* of the C ABI).

    ``problems`` is a list of QP-like objects (see ``Solver``); optional per-instance
    ``x0``/``y0``/``sigma0``/``lambda_A``/``lambda_Q`` lists set warm starts and fixed
    parameters."""

    def __init__(self, problems, stream=None, x0=None, y0=None, sigma0=None, lambda_A=None, lambda_Q=None,
                 torch_alloc=None, **params):
        L = lib()
        keep = []

        def hold(a, dtype):
            if dtype is None:
                keep.append(a)
                return a
            if hasattr(a, "data_ptr"):
                import torch
                tdt = {np.int32: torch.int32, np.float64: torch.float64}[dtype]
                a = a.to(tdt).contiguous()
            else:
                a = np.ascontiguousarray(a, dtype=dtype)
            keep.append(a)
            return a

        p = default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        if stream is not None:
            p.stream = int(stream)
        self._alloc = None
        if torch_alloc is None:
            torch_alloc = _torch_cuda()
        if torch_alloc:   # device memory through PyTorch's caching allocator, as for Solver
            self._alloc = _TorchAllocator()
            p.alloc = self._alloc.alloc
            p.free = self._alloc.free
        self.params = p
        cnt = len(problems)
        arr = (hprqp_problem * cnt)()
        self.ns, self.ms = [], []
        for i, qp in enumerate(problems):
            pr = arr[i]
            pr.n, pr.m = int(qp.n), int(qp.m)
            self.ns.append(int(qp.n))
            self.ms.append(int(qp.m))
            pr.Q = C.pointer(_qop_of(qp, hold))
            if qp.m:
                pr.A_rowptr = _ptr(hold(qp.A_rowptr, np.int32))
                pr.A_colidx = _ptr(hold(qp.A_colidx, np.int32))
                pr.A_vals = _ptr(hold(qp.A_vals, np.float64))
                pr.l = _ptr(hold(qp.l, np.float64))
                pr.u = _ptr(hold(qp.u, np.float64))
            pr.c = _ptr(hold(qp.c, np.float64))
            pr.L = _ptr(hold(qp.L, np.float64)) if qp.L is not None else None
            pr.U = _ptr(hold(qp.U, np.float64)) if qp.U is not None else None
            pr.phi = int(qp.phi)
            pr.lam = float(qp.lam)
            if x0 is not None and x0[i] is not None:
                pr.x0 = _ptr(hold(x0[i], np.float64))
                if y0 is not None and y0[i] is not None and qp.m:
                    pr.y0 = _ptr(hold(y0[i], np.float64))
            pr.sigma0 = float(sigma0[i]) if sigma0 is not None else 0.0
            pr.lambda_A = float(lambda_A[i]) if lambda_A is not None else 0.0
            pr.lambda_Q = float(lambda_Q[i]) if lambda_Q is not None else 0.0
        h = C.c_void_p()
        st = L.hprqp_batch_create(C.byref(h), cnt, arr, C.byref(p))
        keep.clear()
        if st != HPRQP_OK:
            raise HPRQPError(st, L.hprqp_batch_last_error(None).decode())
        self.h = h
        self.count = cnt

    def _check(self, st, ok=(HPRQP_OK,)):
        if st not in ok:
            raise HPRQPError(st, lib().hprqp_batch_last_error(self.h).decode())
        return st

    def solve(self, tol=1e-8, max_iter=1_000_000):
        st = lib().hprqp_batch_solve(self.h, float(tol), int(max_iter))
        self._check(st, ok=(HPRQP_OK, HPRQP_MAX_ITER))
        return STATUS_NAMES[st]

    def get(self, i):
        x = np.empty(self.ns[i])
        y = np.empty(max(self.ms[i], 1))
        z = np.empty(self.ns[i])
        k = hprqp_kkt()
        self._check(lib().hprqp_batch_get(self.h, int(i), _ptr(x), _ptr(y) if self.ms[i] else None, _ptr(z),
                                          C.byref(k)))
        return x, y[:self.ms[i]], z, k.as_dict()

    def stats(self):
        sec = C.c_double()
        n = C.c_int64()
        self._check(lib().hprqp_batch_stats(self.h, C.byref(sec), C.byref(n)))
        return {"seconds": sec.value, "kernel_launches": n.value}

    def schedule(self):
        """Per bucket of instances (by n): the autotuner's block size (threads per instance) and
        shared-memory F copy."""
        out = np.zeros(20, np.int64)
        self._check(lib().hprqp_batch_schedule(self.h, _ptr(out)))
        return [{"n_from": int(out[5 * k]), "instances": int(out[5 * k + 1]), "threads": int(out[5 * k + 2]),
                 "f_in_smem": bool(out[5 * k + 3]), "f_capacity": int(out[5 * k + 4])}
                for k in range(4)]

    def close(self):
        if getattr(self, "h", None):
            lib().hprqp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
