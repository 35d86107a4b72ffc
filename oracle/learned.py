"""CPU FP64 oracle of the learned warm start: TEST INFRASTRUCTURE ONLY.

Plain numpy restatement of what the GPU warm-start path computes, for parity tests.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; it shares no code with the CUDA library.

The paper starts HPR-QP at the origin (Sec. 4.1) and allows any starting point, since the
Halpern step of Algorithm 1 (Step 5) and Algorithm 4 anchors each restart cycle at its first
iterate.  The learned part predicts that starting point.  Its definition (not in the paper):

  features   f = P [c; u]                          (BF16 operands, exact products)
  network    h_0 = bf16(standardised f),  h_{l+1} = bf16(relu(W_l h_l + b_l)),
             o = W_{L-1} h_{L-1} + b_{L-1}          (W_l rounded to BF16)
  decoder    ell = alpha o[1:1+r],  z0 = clip(mu + Phi ell, lo, hi)
  loss       w_sigma/2 (o_0 - s)^2 + ||mu + Phi ell - z*||^2 / (2E), batch mean
  training   backpropagation (chain rule) with the gradients of the hidden layers rounded to
             BF16 where the GPU stores them, and Adam (Kingma and Ba, 2015).

BF16 rounding: FP64 -> FP32 (round to nearest even) -> BF16 (round to nearest even on the
16 dropped bits); non-finite values become 0.  Every matrix product here is a plain
``@`` in FP64.  With ``bf16=False`` the network runs in plain FP64 (used by the
finite-difference pins).
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), via FP32; non-finite -> 0."""
    x = np.asarray(x, dtype=np.float64)
    x = np.where(np.isfinite(x), x, 0.0)
    f = x.astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(x) -> np.ndarray:
    """The uint16 bit patterns of bf16_round(x)."""
    r = bf16_round(x).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b) -> np.ndarray:
    b = np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def _rnd(x, on):
    return bf16_round(x) if on else np.asarray(x, dtype=np.float64)


def mlp_forward(Ws, bs, X, bf16=True):
    """Forward pass.  Ws[l]: (d_{l+1}, d_l), bs[l]: (d_{l+1},), X: (B, d_0) (already
    BF16-valued when bf16).  Returns (output (B, d_L), inputs of every layer)."""
    h = np.asarray(X, dtype=np.float64)
    hs = []
    L = len(Ws)
    for l in range(L):
        hs.append(h)
        z = h @ _rnd(Ws[l], bf16).T + np.asarray(bs[l], dtype=np.float64)
        if l + 1 < L:
            h = _rnd(np.maximum(z, 0.0), bf16)
        else:
            return z, hs
    raise AssertionError("unreachable")


def mlp_backward(Ws, hs, dY, bf16=True):
    """Gradients (dW_l, db_l) of a loss with dL/dY = dY, for the inputs hs of mlp_forward."""
    L = len(Ws)
    dZ = _rnd(dY, bf16)
    gW = [None] * L
    gb = [None] * L
    for l in range(L - 1, -1, -1):
        gW[l] = dZ.T @ hs[l]
        gb[l] = dZ.sum(axis=0)
        if l == 0:
            break
        dX = dZ @ _rnd(Ws[l], bf16)
        dZ = _rnd(dX * (hs[l] > 0), bf16)
    return gW, gb


def adam(W, m, v, g, t, lr, beta1, beta2, eps):
    """One Adam step; returns the new (W, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return W - lr * mhat / (np.sqrt(vhat) + eps), m, v


def ws_loss(O, G, R, dd, s, alpha, E, w_sigma, r, s_mean=0.0, s_istd=1.0):
    """Warm-start loss of a batch and its gradient w.r.t. O (see the module docstring).
    O: (B, >= 1 + r); G = Phi^T Phi (r, r); R = Phi^T (z* - mu) per instance, (r, B);
    dd = ||z* - mu||^2 (B,); s: log sigma targets (B,), standardised as (s - s_mean) s_istd.
    Returns (dO, sigma part, latent part)."""
    O = np.asarray(O, dtype=np.float64)
    B = O.shape[0]
    o = O[:, 1:1 + r]
    Go = o @ G.T
    e0 = O[:, 0] - (np.asarray(s, dtype=np.float64) - s_mean) * s_istd
    dO = np.zeros_like(O)
    dO[:, 0] = w_sigma * e0 / B
    dO[:, 1:1 + r] = (alpha * alpha * Go - alpha * R.T) / E / B
    quad = np.einsum("bk,bk->b", o, Go)
    lin = np.einsum("bk,kb->b", o, R)
    lat = 0.5 * (alpha * alpha * quad - 2.0 * alpha * lin + dd) / E
    return dO, float(np.mean(0.5 * w_sigma * e0 * e0)), float(np.mean(lat))


def decode(Phi, mu, ell, alpha, lo, hi):
    """z0[b] = clip(mu + alpha Phi ell[b], lo, hi) for each row of ell (B, r)."""
    # (the GPU decoder rounds ell to BF16 first: pass bf16_round(O[:, 1:1+r]) for parity)
    Z = mu[None, :] + alpha * (np.asarray(ell, dtype=np.float64) @ np.asarray(Phi, dtype=np.float64).T)
    return np.clip(Z, lo[None, :], hi[None, :])


def sigma0(O, s_mean, s_istd):
    """Initial penalty parameter from column 0 of the network output."""
    return np.exp(s_mean + np.asarray(O, dtype=np.float64)[:, 0] / s_istd)


def standardize(F, mean, istd):
    """bf16((F - mean) * istd) for feature-major F (d, B); returns batch-major (B, d)."""
    return bf16_round(((F - mean[:, None]) * istd[:, None]).T)


def row_stats(F, floor):
    """Row means and 1/sqrt(max(population variance, floor))."""
    F = np.asarray(F, dtype=np.float64)
    mu = F.mean(axis=1)
    var = ((F - mu[:, None]) ** 2).mean(axis=1)
    return mu, 1.0 / np.sqrt(np.maximum(var, floor))
