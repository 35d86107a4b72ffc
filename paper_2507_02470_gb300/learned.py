"""Learned warm start for a parametric family of HPR-QP problems (binding of hprqp_learn.h).

A family shares A, Q and the box C and varies c and the row bounds.  ``LearnedWarmStart``
holds the fixed random projection P (d0 x D, D = n + m), the fixed decoder basis Phi
(D x r), the mean training solution mu, the feature statistics and a BF16 multilayer
perceptron; ``fit`` trains it on solutions produced by ``Solver`` and ``predict`` returns
starting points (x0, y0) and initial penalties sigma0 for new members.  Every arithmetic step
runs in the library's CUDA kernels (tcgen05 GEMMs, conversions, loss, Adam, decoder); this
module allocates device buffers with PyTorch and passes pointers.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

from ._lib import HPRQPError, lib

def _torch():
    import torch
    return torch


def _chk(st):
    if st != 0:
        raise HPRQPError(st, lib().hprqp_learn_last_error().decode())


def _sp(stream):
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def round8(x: int) -> int:
    return (int(x) + 7) // 8 * 8


def auto_splits(M, N, K, device=None):
    """K-splits that give about one CTA per SM (the library's tile rule: 128 x BN tiles with
    BN = 64, 128 or 256 by N)."""
    torch = _torch()
    sms = torch.cuda.get_device_properties(device or torch.cuda.current_device()).multi_processor_count
    bn = 64 if N <= 64 else 128 if N < 512 else 256
    tiles = -(-M // 128) * -(-N // bn)
    kb = -(-K // 64)
    return int(max(1, min(kb, round(sms / tiles))))


def gemm_bf16(A, B, out=None, splits=0, stream=None):
    """out (M x N, FP32) = A @ B^T for CUDA bfloat16 tensors A (M x K) and B (N x K) whose rows
    are contiguous (any row stride that is a multiple of 8).  splits <= 0: ``auto_splits``."""
    torch = _torch()
    M, K = A.shape
    N, K2 = B.shape
    if K2 != K or A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("A (M x K) and B (N x K) need unit column stride")
    if splits <= 0:
        splits = auto_splits(M, N, K, A.device)
    if out is None:
        out = torch.empty(M, N, dtype=torch.float32, device=A.device)
    work = None
    if splits > 1:
        work = torch.empty(splits * M * N, dtype=torch.float32, device=A.device)
    _chk(lib().hprqp_gemm_bf16(M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), out.data_ptr(),
                               out.stride(0), int(splits), None if work is None else work.data_ptr(), _sp(stream)))
    return out


def check():
    """Raises if a GEMM kernel gave up a bounded wait since the last check."""
    _chk(lib().hprqp_learn_check())


def cast_bf16(x, sub=None, scale=1.0, ld=None, rownorm2=None, stream=None):
    """bf16((x - sub) * scale) of a 2-D CUDA float64/float32 tensor (rows x cols) into a new
    rows x ld bfloat16 tensor (padding zero); returns it (and fills rownorm2 if given)."""
    torch = _torch()
    rows, cols = x.shape
    ld = round8(cols) if ld is None else ld
    out = torch.empty(rows, ld, dtype=torch.bfloat16, device=x.device)
    f = lib().hprqp_cast_bf16_f64 if x.dtype == torch.float64 else lib().hprqp_cast_bf16_f32
    if x.dtype not in (torch.float64, torch.float32) or x.stride(1) != 1:
        raise ValueError("x must be float64/float32 with unit column stride")
    _chk(f(x.data_ptr(), rows, cols, x.stride(0), None if sub is None else sub.data_ptr(), float(scale),
           out.data_ptr(), ld, None if rownorm2 is None else rownorm2.data_ptr(), _sp(stream)))
    return out


class MLP:
    """BF16 multilayer perceptron with ReLU hidden layers, trained with Adam (hprqp_mlp_*)."""

    def __init__(self, dims, max_batch, stream=None):
        self.dims = [int(d) for d in dims]
        self.L = len(self.dims) - 1
        self.max_batch = int(max_batch)
        self.stream = stream
        arr = (C.c_int32 * len(self.dims))(*self.dims)
        h = C.c_void_p()
        _chk(lib().hprqp_mlp_create(C.byref(h), self.L, arr, self.max_batch, _sp(stream)))
        self.h = h
        self.t = 0

    def set_layer(self, l, W, b):
        W = np.ascontiguousarray(W, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        assert W.shape == (self.dims[l + 1], self.dims[l]) and b.shape == (self.dims[l + 1],)
        _chk(lib().hprqp_mlp_set_layer(self.h, l, W.ctypes.data, b.ctypes.data))

    def get_layer(self, l):
        W = np.empty((self.dims[l + 1], self.dims[l]), dtype=np.float32)
        b = np.empty(self.dims[l + 1], dtype=np.float32)
        _chk(lib().hprqp_mlp_get_layer(self.h, l, W.ctypes.data, b.ctypes.data))
        return W, b

    def get_grad(self, l):
        W = np.empty((self.dims[l + 1], self.dims[l]), dtype=np.float32)
        b = np.empty(self.dims[l + 1], dtype=np.float32)
        _chk(lib().hprqp_mlp_get_grad(self.h, l, W.ctypes.data, b.ctypes.data))
        return W, b

    def forward(self, X, out=None):
        """X: CUDA bfloat16 (B x >= dims[0], row stride multiple of 8) -> FP32 (B x dims[-1])."""
        torch = _torch()
        B = X.shape[0]
        if out is None:
            out = torch.empty(B, self.dims[-1], dtype=torch.float32, device=X.device)
        _chk(lib().hprqp_mlp_forward(self.h, X.data_ptr(), X.stride(0), B, out.data_ptr(), out.stride(0)))
        return out

    def backward(self, dY):
        _chk(lib().hprqp_mlp_backward(self.h, dY.data_ptr(), dY.stride(0)))

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        _chk(lib().hprqp_mlp_adam(self.h, float(lr), float(beta1), float(beta2), float(eps), self.t))

    def close(self):
        if getattr(self, "h", None):
            lib().hprqp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rows(Cs, Us):
    return lambda b0, b1: (Cs[b0:b1], Us[b0:b1])


def dual_box(l, u):
    """Sign box of the multipliers y of l <= Ax <= u in the solver's convention (y <= 0 on rows
    with l = -inf, y >= 0 on rows with u = +inf, free on rows with both bounds finite)."""
    l = np.asarray(l, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lo = np.where(np.isfinite(u), -np.inf, 0.0)
    hi = np.where(np.isfinite(l), np.inf, 0.0)
    return lo, hi


@dataclass
class FitReport:
    epochs: int
    loss_sigma: List[float] = field(default_factory=list)
    loss_latent: List[float] = field(default_factory=list)
    latent_baseline: float = 0.0      # latent loss of ell = 0 (decoding to mu)
    seconds: float = 0.0              # whole fit (targets, features, statistics, training)
    train_seconds: float = 0.0        # the Adam steps alone
    steps: int = 0


class LearnedWarmStart:
    """Learned (x0, y0, sigma0) for members of one problem family (fixed A, Q, C; varying c, u).

    n, m: sizes; L, U: the box C; l, u: row bounds of the nominal member (their finiteness
    fixes the sign box of y).  d0, hidden, r: feature width, hidden widths, latent width.
    """

    def __init__(self, n, m, L, U, l, u, d0=512, hidden=(1024, 1024), r=256, seed=0, max_batch=256,
                 stream=None, device="cuda", chunk=512):
        torch = _torch()
        self.n, self.m, self.D = int(n), int(m), int(n) + int(m)
        self.Dp = round8(self.D)
        self.d0, self.r = int(d0), int(r)
        self.dims = [self.d0, *[int(h) for h in hidden], 1 + self.r]
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.chunk = int(chunk)
        self.max_batch = int(max_batch)
        import qpgen
        # fixed random matrices: P ~ N(0, 1/D) (d0 x D), Phi ~ N(0, 1/r) (D x r) and Phi^T
        P = torch.from_numpy(qpgen.ws_gaussian(self.d0, self.D, seed + 11)).to(self.device)
        self.P = cast_bf16(P, scale=1.0 / math.sqrt(self.D), ld=self.Dp, stream=self.stream)
        del P
        Phi = qpgen.ws_gaussian(self.D, self.r, seed + 12)
        Pt = torch.from_numpy(Phi).to(self.device)
        self.Phi = cast_bf16(Pt, scale=1.0 / math.sqrt(self.r), ld=round8(self.r), stream=self.stream)
        Pt = torch.from_numpy(np.ascontiguousarray(Phi.T)).to(self.device)
        self.PhiT = cast_bf16(Pt, scale=1.0 / math.sqrt(self.r), ld=self.Dp, stream=self.stream)
        del Pt, Phi
        self.alpha = math.sqrt(self.r / self.D)       # unit-norm columns of alpha * Phi
        self.E = float(self.D)                        # latent loss = mean squared error / 2
        ylo, yhi = dual_box(l, u)
        lo = np.concatenate([np.asarray(L, dtype=np.float64), ylo])
        hi = np.concatenate([np.asarray(U, dtype=np.float64), yhi])
        self.lo = torch.from_numpy(lo).to(self.device)
        self.hi = torch.from_numpy(hi).to(self.device)
        self.mlp = MLP(self.dims, self.max_batch, stream=self.stream)
        rng = np.random.default_rng(seed + 13)
        for li in range(len(self.dims) - 1):
            din, dout = self.dims[li], self.dims[li + 1]
            std = math.sqrt(2.0 / din) if li + 2 < len(self.dims) else 0.01 / math.sqrt(din)
            self.mlp.set_layer(li, rng.standard_normal((dout, din)) * std, np.zeros(dout))
        self.mu = None
        self.fmean = self.fistd = None
        self.s_mean = 0.0
        self.s_istd = 1.0

    # ---------------------------------------------------------------- data preparation
    def _pack(self, Cs, Us):
        """[c; u] rows (B x D) as BF16 (B x Dp) on the device."""
        torch = _torch()
        B = Cs.shape[0]
        cu = torch.empty(B, self.D, dtype=torch.float64, device=self.device)
        cu[:, :self.n].copy_(torch.as_tensor(Cs, dtype=torch.float64), non_blocking=False)
        cu[:, self.n:].copy_(torch.as_tensor(Us, dtype=torch.float64), non_blocking=False)
        return cast_bf16(cu, ld=self.Dp, stream=self.stream)

    def raw_features(self, data, N, out=None):
        """F (d0 x N, FP32 feature-major) = P [c; u] for members 0..N-1, where data(b0, b1)
        returns their (c, u) rows as (b1-b0) x n and (b1-b0) x m arrays."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.d0, N, dtype=torch.float32, device=self.device)
        for b0 in range(0, N, self.chunk):
            b1 = min(N, b0 + self.chunk)
            Cs, Us = data(b0, b1)
            cu = self._pack(Cs, Us)
            gemm_bf16(self.P, cu, out=out[:, b0:b1], stream=self.stream)
        return out

    def features(self, Cs, Us):
        """Standardised BF16 features (B x round8(d0)) with the training statistics."""
        torch = _torch()
        F = self.raw_features(_rows(Cs, Us), Cs.shape[0])
        B = F.shape[1]
        X = torch.zeros(B, round8(self.d0), dtype=torch.bfloat16, device=self.device)
        _chk(lib().hprqp_ws_standardize(F.data_ptr(), self.d0, B, F.stride(0), self.fmean.data_ptr(),
                                        self.fistd.data_ptr(), X.data_ptr(), X.stride(0), _sp(self.stream)))
        return X

    # ---------------------------------------------------------------- training
    def fit(self, data, Z, sigma, epochs=30, batch=256, lr=1e-3, w_sigma=1.0, log=None):
        """data: (Cs, Us) arrays (N x n, N x m) of the training members, or a function
        data(b0, b1) returning rows b0..b1-1 of them; Z (N x D, FP64 CUDA): their solutions
        (x, y); sigma (N,): the final sigma of each solve."""
        import time
        torch = _torch()
        t0 = time.perf_counter()
        N = Z.shape[0]
        if isinstance(data, tuple):
            data = _rows(*data)
        s = self.stream
        self.mu = torch.empty(self.D, dtype=torch.float64, device=self.device)
        _chk(lib().hprqp_col_mean_f64(Z.data_ptr(), N, self.D, Z.stride(0), self.mu.data_ptr(), _sp(s)))
        # R = Phi^T (z* - mu) (r x N) and dd = ||z* - mu||^2, in chunks
        self.R = torch.empty(self.r, N, dtype=torch.float32, device=self.device)
        self.dd = torch.empty(N, dtype=torch.float64, device=self.device)
        for b0 in range(0, N, self.chunk):
            b1 = min(N, b0 + self.chunk)
            dz = cast_bf16(Z[b0:b1], sub=self.mu, ld=self.Dp, rownorm2=self.dd[b0:b1], stream=s)
            gemm_bf16(self.PhiT, dz, out=self.R[:, b0:b1], stream=s)
            del dz
        # G = Phi^T Phi
        self.G = gemm_bf16(self.PhiT, self.PhiT, stream=s)
        # features and their statistics
        F = self.raw_features(data, N)
        self.fmean = torch.empty(self.d0, dtype=torch.float32, device=self.device)
        self.fistd = torch.empty(self.d0, dtype=torch.float32, device=self.device)
        _chk(lib().hprqp_row_stats(F.data_ptr(), self.d0, N, F.stride(0), C.c_float(1e-20), self.fmean.data_ptr(),
                                   self.fistd.data_ptr(), _sp(s)))
        X = torch.zeros(N, round8(self.d0), dtype=torch.bfloat16, device=self.device)
        _chk(lib().hprqp_ws_standardize(F.data_ptr(), self.d0, N, F.stride(0), self.fmean.data_ptr(),
                                        self.fistd.data_ptr(), X.data_ptr(), X.stride(0), _sp(s)))
        del F
        # log sigma targets and their statistics
        ls = torch.as_tensor(np.log(np.asarray(sigma, dtype=np.float64)), dtype=torch.float32).to(self.device)
        sm = torch.empty(1, dtype=torch.float32, device=self.device)
        si = torch.empty(1, dtype=torch.float32, device=self.device)
        _chk(lib().hprqp_row_stats(ls.data_ptr(), 1, N, N, C.c_float(1e-6), sm.data_ptr(), si.data_ptr(), _sp(s)))
        self.s_mean, self.s_istd = float(sm.item()), float(si.item())
        # training
        rep = FitReport(epochs=epochs)
        rep.latent_baseline = float(self.dd.mean().item()) / (2.0 * self.E)
        B = min(batch, self.max_batch)
        dO = torch.zeros(B, self.dims[-1], dtype=torch.float32, device=self.device)
        loss = torch.zeros(2, dtype=torch.float32, device=self.device)
        torch.cuda.synchronize()
        t_train = time.perf_counter()
        for ep in range(epochs):
            acc = torch.zeros(2, dtype=torch.float64, device=self.device)
            nb = 0
            for b0 in range(0, N - B + 1, B):
                O = self.mlp.forward(X[b0:b0 + B])
                _chk(lib().hprqp_ws_loss(O.data_ptr(), O.stride(0), B, self.r, self.G.data_ptr(),
                                         self.R[:, b0:].data_ptr(), self.R.stride(0), self.dd[b0:].data_ptr(),
                                         ls[b0:].data_ptr(), C.c_float(self.s_mean), C.c_float(self.s_istd),
                                         C.c_float(self.alpha), C.c_float(self.E), C.c_float(w_sigma),
                                         dO.data_ptr(), dO.stride(0), self.dims[-1], loss.data_ptr(), _sp(s)))
                self.mlp.backward(dO)
                self.mlp.adam(lr=lr)
                acc += loss.double()
                nb += 1
            acc = (acc / max(nb, 1)).tolist()
            rep.loss_sigma.append(acc[0])
            rep.loss_latent.append(acc[1])
            if log:
                log(f"epoch {ep}: sigma {acc[0]:.4g} latent {acc[1]:.4g} (mu only {rep.latent_baseline:.4g})")
        check()
        rep.train_seconds = time.perf_counter() - t_train
        rep.steps = self.mlp.t
        rep.seconds = time.perf_counter() - t0
        return rep

    # ---------------------------------------------------------------- inference
    def predict(self, Cs, Us):
        """(Z0 (B x D) FP64 CUDA, sigma0 (B,) FP64 CUDA) for new members."""
        torch = _torch()
        B = Cs.shape[0]
        Z0 = torch.empty(B, self.D, dtype=torch.float64, device=self.device)
        sig = torch.empty(B, dtype=torch.float64, device=self.device)
        X = self.features(Cs, Us)
        for b0 in range(0, B, self.max_batch):
            b1 = min(B, b0 + self.max_batch)
            O = self.mlp.forward(X[b0:b1])
            work = torch.empty(self.D * (b1 - b0), dtype=torch.float32, device=self.device)
            _chk(lib().hprqp_ws_decode(self.Phi.data_ptr(), self.Phi.stride(0), self.D, self.r, O.data_ptr(),
                                       O.stride(0), b1 - b0, C.c_float(self.alpha), C.c_float(self.s_mean),
                                       C.c_float(self.s_istd), self.mu.data_ptr(), self.lo.data_ptr(),
                                       self.hi.data_ptr(), work.data_ptr(), Z0[b0:b1].data_ptr(), Z0.stride(0),
                                       sig[b0:b1].data_ptr(), _sp(self.stream)))
        return Z0, sig

    # ---------------------------------------------------------------- persistence
    def save(self, path, **meta):
        """Everything inference needs, in one .npz: the layers' weights as BF16 bits (the
        forward pass multiplies BF16 weights, so nothing it uses is lost), the biases, the mean
        training solution mu, the feature and log-sigma statistics, and `meta` (e.g. the family
        and the training set it came from)."""
        arrs = {"dims": np.asarray(self.dims, np.int64), "n": self.n, "m": self.m,
                "mu": self.mu.cpu().numpy(), "fmean": self.fmean.cpu().numpy(), "fistd": self.fistd.cpu().numpy(),
                "s_mean": self.s_mean, "s_istd": self.s_istd}
        for li in range(len(self.dims) - 1):
            W, b = self.mlp.get_layer(li)
            arrs[f"W{li}"] = bf16_bits_rne(W)
            arrs[f"b{li}"] = b
        for k, v in meta.items():
            arrs["meta_" + k] = np.asarray(v)
        np.savez_compressed(path, **arrs)

    def load(self, path):
        """The state written by save() (same sizes and seed); returns its meta entries."""
        torch = _torch()
        z = np.load(path)
        if list(z["dims"]) != self.dims or int(z["n"]) != self.n or int(z["m"]) != self.m:
            raise ValueError(f"{path}: network of another shape")
        for li in range(len(self.dims) - 1):
            W = (z[f"W{li}"].astype(np.uint32) << 16).view(np.float32)
            self.mlp.set_layer(li, W, z[f"b{li}"])
        self.mu = torch.from_numpy(z["mu"]).to(self.device)
        self.fmean = torch.from_numpy(z["fmean"]).to(self.device)
        self.fistd = torch.from_numpy(z["fistd"]).to(self.device)
        self.s_mean, self.s_istd = float(z["s_mean"]), float(z["s_istd"])
        return {k[5:]: z[k] for k in z.files if k.startswith("meta_")}

    def close(self):
        self.mlp.close()


def bf16_bits_rne(a):
    """float32 array -> BF16 bit patterns (uint16), rounded to nearest, ties to even."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def solve_members(base, data, N, stream=None, Z=None, starts=None, lam=None, tol=1e-8, workers=1,
                  fallback=True):
    """Solves members 0..N-1 of a family with the plain solver (one handle per worker thread,
    each on its own CUDA stream).  data(b0, b1) -> (Cs, Us) as in ``LearnedWarmStart.fit``;
    starts: optional (Z0 (N x D) host/CUDA, sigma0 (N,)) warm starts; lam: (lambda_A,
    lambda_Q) to skip the power method.  With ``fallback`` a member whose warm start is
    rejected (non-finite) or whose warm-started solve does not converge is solved again from
    the origin (counted in "fallbacks").  Writes solutions into Z (N x D, CUDA) if given and
    returns a dict of per-member iterations, seconds, objectives, final sigmas, the lambdas
    used and the fallback count."""
    import threading
    import time
    import torch
    from ._lib import Solver
    n, m = base.n, base.m
    out = {"iters": np.zeros(N, dtype=np.int64), "seconds": np.zeros(N), "pobj": np.zeros(N),
           "sigma": np.zeros(N), "status": [""] * N, "fallbacks": 0}
    lam_box = [lam]
    lock = threading.Lock()
    errors = []

    def work(wid):
        try:
            st_ = torch.cuda.Stream() if workers > 1 else None
            sp = st_.cuda_stream if st_ is not None else stream
            with Solver(base, stream=sp) as s:
                if lam_box[0] is not None:
                    s.set_lambda(*lam_box[0])
                for b0 in range(wid, N, workers):
                    Cs, Us = data(b0, b0 + 1)
                    s.set_data(c=Cs[0], u=Us[0])
                    t0 = time.perf_counter()
                    warm_ok = starts is not None
                    if warm_ok:
                        z0, sg = starts
                        try:
                            s.set_warm_start(z0[b0, :n], z0[b0, n:], float(sg[b0]))
                        except HPRQPError:
                            if not fallback:
                                raise
                            warm_ok = False
                    if not warm_ok:
                        s.set_warm_start(None, None, 0.0)
                    status = s.solve(tol=tol)
                    if starts is not None and fallback and (not warm_ok or status != "converged"):
                        if warm_ok:                     # the warm-started solve failed: cold
                            s.set_warm_start(None, None, 0.0)
                            status = s.solve(tol=tol)
                        with lock:
                            out["fallbacks"] += 1
                    dt = time.perf_counter() - t0
                    if Z is not None:
                        _, _, _, _, k = s.get(Z[b0, :n], Z[b0, n:], None, None)
                    else:
                        k = s.kkt()
                    out["iters"][b0] = k["iters"]
                    out["seconds"][b0] = dt
                    out["pobj"][b0] = k["pobj"]
                    out["sigma"][b0] = k["sigma"]
                    out["status"][b0] = status
                    with lock:
                        if lam_box[0] is None:
                            lam_box[0] = (k["lambda_A"], k["lambda_Q"])
                    s.set_lambda(*lam_box[0])
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    if workers > 1 and lam_box[0] is None:
        # the first member fixes lambda_A, lambda_Q for every worker
        first = solve_members(base, data, 1, stream=stream, Z=Z, starts=starts, lam=None, tol=tol)
        lam_box[0] = first["lambda"]
    threads = [threading.Thread(target=work, args=(w,)) for w in range(workers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    out["lambda"] = lam_box[0]
    return out
