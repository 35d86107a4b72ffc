"""SpMV timing comparison: cuSPARSE CSR SpMV against the solver's fused A and A^T passes.

    python -m paper_2507_02470_gb300.spmv_compare --workload c1

The paper runs its sparse products with cuSPARSE (CSR_ALG2, Sec. 3.1 remark on
implementation).  This tool times cusparseSpMV (CSR_ALG1 and CSR_ALG2, FP64) for y = A x and
x = A^T y on the workload's A and its stored transpose, with L2 flushed before every timed
call, and the solver's own passes that contain those products (K3: A v plus the y-step and
Halpern update; K4: A^T ybar plus the wbar update) from hprqp_profile inside real iterations.
cuSPARSE is called through ctypes for this comparison only; the solver never uses it.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import sys

import numpy as np

# cuSPARSE enum values (cusparse.h, library_types.h)
_INDEX_32I = 2
_BASE_ZERO = 0
_R_64F = 1
_OP_N = 0
_ALGS = {"csr_alg1": 2, "csr_alg2": 3}


def _cusparse():
    for name in ("libcusparse.so.12", "libcusparse.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcusparse.so")
    return C.CDLL(cand)


def _ok(st, what):
    if st != 0:
        raise RuntimeError(f"{what} failed with cuSPARSE status {st}")


class CsrSpMV:
    """y = M x with cuSPARSE for one CSR matrix on the device (torch tensors)."""

    def __init__(self, lib, handle, rows, cols, rp, ci, va, x, y):
        self.lib, self.h = lib, handle
        self.mat, self.vx, self.vy = C.c_void_p(), C.c_void_p(), C.c_void_p()
        _ok(lib.cusparseCreateCsr(C.byref(self.mat), C.c_int64(rows), C.c_int64(cols), C.c_int64(int(ci.numel())),
                                  C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()), C.c_void_p(va.data_ptr()),
                                  _INDEX_32I, _INDEX_32I, _BASE_ZERO, _R_64F), "cusparseCreateCsr")
        _ok(lib.cusparseCreateDnVec(C.byref(self.vx), C.c_int64(cols), C.c_void_p(x.data_ptr()), _R_64F), "DnVec x")
        _ok(lib.cusparseCreateDnVec(C.byref(self.vy), C.c_int64(rows), C.c_void_p(y.data_ptr()), _R_64F), "DnVec y")
        self.alpha = C.c_double(1.0)
        self.beta = C.c_double(0.0)
        self.buf = {}

    def prepare(self, alg):
        import torch
        sz = C.c_size_t(0)
        _ok(self.lib.cusparseSpMV_bufferSize(self.h, _OP_N, C.byref(self.alpha), self.mat, self.vx,
                                             C.byref(self.beta), self.vy, _R_64F, _ALGS[alg], C.byref(sz)),
            "cusparseSpMV_bufferSize")
        self.buf[alg] = torch.empty(max(int(sz.value), 16), dtype=torch.uint8, device="cuda")

    def run(self, alg):
        _ok(self.lib.cusparseSpMV(self.h, _OP_N, C.byref(self.alpha), self.mat, self.vx, C.byref(self.beta),
                                  self.vy, _R_64F, _ALGS[alg], C.c_void_p(self.buf[alg].data_ptr())),
            "cusparseSpMV")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c1", choices=["c1", "c4"],
                    help="c1: A of the CQP n=1e6, m=5e5; c4: A of the CQP n=1e5, m=5e4")
    ap.add_argument("--reps", type=int, default=30)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import scipy.sparse as sp
    import torch
    import qpgen
    import paper_2507_02470_gb300 as pkg
    pkg.build()
    qp = (qpgen.large_cqp(n=1_000_000, m=500_000, seed=0) if args.workload == "c1"
          else qpgen.param_family_base(n=100_000, m=50_000, seed=0))
    n, m = qp.n, qp.m
    A = sp.csr_matrix((qp.A_vals, qp.A_colidx, qp.A_rowptr), shape=(m, n))
    AT = A.T.tocsr()
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    mats = {"A": (m, n, dev(A.indptr, np.int32), dev(A.indices, np.int32), dev(A.data, np.float64)),
            "AT": (n, m, dev(AT.indptr, np.int32), dev(AT.indices, np.int32), dev(AT.data, np.float64))}
    xs = {"A": torch.randn(n, dtype=torch.float64, device="cuda"),
          "AT": torch.randn(m, dtype=torch.float64, device="cuda")}
    ys = {"A": torch.empty(m, dtype=torch.float64, device="cuda"),
          "AT": torch.empty(n, dtype=torch.float64, device="cuda")}
    lib = _cusparse()
    h = C.c_void_p()
    _ok(lib.cusparseCreate(C.byref(h)), "cusparseCreate")
    stream = torch.cuda.current_stream()
    _ok(lib.cusparseSetStream(h, C.c_void_p(stream.cuda_stream)), "cusparseSetStream")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    out = {"workload": args.workload, "n": n, "m": m, "nnz": int(A.nnz), "cusparse_us": {}, "cusparse_GBs": {}}
    for key, (rows, cols, rp, ci, va) in mats.items():
        op = CsrSpMV(lib, h, rows, cols, rp, ci, va, xs[key], ys[key])
        ref = (A if key == "A" else AT) @ xs[key].cpu().numpy()
        alg_bytes = 12 * int(A.nnz) + 4 * (rows + 1) + 8 * (cols + rows)
        for alg in _ALGS:
            op.prepare(alg)
            for _ in range(3):
                op.run(alg)
            torch.cuda.synchronize()
            assert np.allclose(ys[key].cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
            ts = []
            for _ in range(args.reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                op.run(alg)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3)
            us = float(np.median(ts))
            out["cusparse_us"][f"{key}_{alg}"] = round(us, 2)
            out["cusparse_GBs"][f"{key}_{alg}"] = round(alg_bytes / (us * 1e-6) / 1e9, 1)
    lib.cusparseDestroy(h)
    # the solver's fused passes inside real iterations (working set larger than L2)
    with pkg.Solver(qp, launch_mode=2) as s:
        s.solve(tol=1e-30, max_iter=20)
        ms = s.profile(iters=args.reps)
    out["fused_us"] = {"K3 (A v + y-step)": round(ms["a1"] * 1e3, 2), "K4 (A^T ybar + wbar)": round(ms["at"] * 1e3, 2)}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
