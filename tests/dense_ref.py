"""Dense, definition-level helpers for pinning the oracle on tiny problems (n <= 8).

Everything here is written from the definitions in the paper (arXiv 2507.02470), not from
the simplified update formulas the oracle uses, so that agreement is evidence:
  * ``brute_force``: exact KKT points of the CCQP by enumerating active sets.
  * ``metric_M``: the operator M of eq. (2.12) assembled block by block from eqs.
    (2.3), (2.6), (2.7), (2.8) and (3.4), with S_sGS taken from its definition (the
    inverse on W = Range(Q) through an eigendecomposition).
  * ``alg2_*``: Algorithm 2 with every w-update solved as a minimisation over W.
"""
from __future__ import annotations

import itertools

import numpy as np


def dense_of(qp):
    A = qp.A_scipy().toarray() if qp.m else np.zeros((0, qp.n))
    Q = qp.Q_scipy().toarray()
    return A, Q


# ------------------------------------------------------------------------- brute force
def _kkt_solve(H, g, G, h):
    """min 1/2 x'Hx + g'x s.t. G x = h via the KKT system (lstsq for singular H)."""
    n = H.shape[0]
    k = G.shape[0]
    K = np.zeros((n + k, n + k))
    K[:n, :n] = H
    K[:n, n:] = G.T
    K[n:, :n] = G
    rhs = np.concatenate([-g, h])
    sol, *_ = np.linalg.lstsq(K, rhs, rcond=None)
    if np.linalg.norm(K @ sol - rhs) > 1e-9 * (1 + np.linalg.norm(rhs)):
        return None, None
    return sol[:n], sol[n:]


def brute_force(qp, tol=1e-9):
    """Optimal value and one KKT point (x, y, z) of a tiny box-phi CQP.

    Inequalities: l <= Ax <= u (rows), L <= x <= U.  Each one is inactive, at its lower or
    at its upper value; every combination is solved as an equality-constrained QP and
    kept when it is primal feasible and the multipliers have the right signs.  y and z
    follow the paper's sign convention  Q x + c = A^* y + z  with y_i >= 0 at a lower
    bound and y_i <= 0 at an upper bound (Sec. 2, eq. (2.1)).
    """
    assert qp.phi == 0
    A, Q = dense_of(qp)
    n, m = qp.n, qp.m
    rows = [(A[i], qp.l[i], qp.u[i]) for i in range(m)] + [(np.eye(n)[j], qp.L[j], qp.U[j]) for j in range(n)]
    best = None
    for states in itertools.product((0, 1, 2), repeat=len(rows)):
        G, h, sign, idx = [], [], [], []
        ok = True
        for r, st in enumerate(states):
            a, lo, hi = rows[r]
            if st == 0:
                if lo == hi:  # equality must be active
                    ok = False
                    break
                continue
            b = lo if st == 1 else hi
            if not np.isfinite(b) or (st == 2 and lo == hi):
                ok = False
                break
            G.append(a); h.append(b); sign.append(1.0 if st == 1 else -1.0); idx.append(r)
        if not ok:
            continue
        G = np.array(G).reshape(-1, n)
        x, lam = _kkt_solve(Q, qp.c, G, np.array(h))
        if x is None:
            continue
        # feasibility
        Ax = A @ x
        if m and (np.any(Ax < qp.l - tol) or np.any(Ax > qp.u + tol)):
            continue
        if np.any(x < qp.L - tol) or np.any(x > qp.U + tol):
            continue
        # Hx + g + G' lam = 0  ->  Qx + c = -G' lam; multipliers of ">= lo" rows must be
        # -lam >= 0, of "<= hi" rows -lam <= 0.
        mult = -lam
        good = True
        for s, mu, r in zip(sign, mult, idx):
            a, lo, hi = rows[r]
            if lo == hi:
                continue
            if s * mu < -1e-8:
                good = False
                break
        if not good:
            continue
        obj = 0.5 * x @ Q @ x + qp.c @ x
        if best is None or obj < best[0] - 1e-12:
            y = np.zeros(m)
            z = np.zeros(n)
            for mu, r in zip(mult, idx):
                if r < m:
                    y[r] += mu
                else:
                    z[r - m] += mu
            best = (obj, x, y, z)
    return best


# ------------------------------------------------------------------------- metric M
def range_basis(Q, tol=1e-10):
    d, V = np.linalg.eigh(Q)
    keep = d > tol * max(1.0, d.max(initial=0.0))
    return d[keep], V[:, keep]


def metric_M(A, Q, sigma, lamA, lamQ):
    """Dense M of eq. (2.12) on (y, w, z, x) in R^m x R^n x R^n x R^n."""
    m, n = A.shape
    AQ = np.hstack([A.T, -Q])                                   # A_Q = [A^*, -Q]  (n x (m+n))
    Sy = lamA * np.eye(m) - A @ A.T                             # eq. (3.4)
    Sw = Q @ (lamQ * np.eye(n) - Q)                             # eq. (2.8) S_w
    S = sigma * np.block([[Sy, np.zeros((m, n))], [np.zeros((n, m)), Sw]])   # eq. (2.6)
    d, V = range_basis(Q)
    # (sigma Q^2 + Q + sigma S_w)^{-1} on W = Range(Q)
    core = sigma * Q @ Q + Q + sigma * Sw
    Winv = V @ np.linalg.inv(V.T @ core @ V) @ V.T if d.size else np.zeros((n, n))
    S1 = sigma ** 2 * A @ Q @ Winv @ Q @ A.T                    # eq. (2.7)
    SsGS = np.block([[S1, np.zeros((m, n))], [np.zeros((n, m)), np.zeros((n, n))]])
    top = sigma * AQ.T @ AQ + S + SsGS
    N = m + 3 * n
    M = np.zeros((N, N))
    yw = slice(0, m + n)
    xs = slice(m + 2 * n, N)
    M[yw, yw] = top
    M[yw, xs] = AQ.T
    M[xs, yw] = AQ
    M[xs, xs] = np.eye(n) / sigma
    return M


def mnorm2_dense(A, Q, sigma, lamA, lamQ, dy, dw, dx):
    n = Q.shape[0]
    v = np.concatenate([dy, dw, np.zeros(n), dx])
    return v @ metric_M(A, Q, sigma, lamA, lamQ) @ v


# ------------------------------------------------------------------------- Algorithm 2
def prox_box(r, L, U):
    return np.minimum(np.maximum(r, L), U)


def alg2_w_update(A, Q, c, sigma, lamQ, y, zb, xb, wk):
    """argmin_{w in W} L_sigma(y, w, zb; xb) + sigma/2 ||w - wk||^2_{S_w}, W = Range(Q),
    solved as an unconstrained quadratic in the coordinates of an orthonormal basis of W."""
    d, V = range_basis(Q)
    n = Q.shape[0]
    if d.size == 0:
        return np.zeros(n)
    Sw = Q @ (lamQ * np.eye(n) - Q)
    QV = Q @ V
    g0 = A.T @ y + zb - c
    # objective in a: 1/2 a'V'QVa - xb'QVa + sigma/2 ||-QVa + g0||^2 + sigma/2 (Va-wk)'Sw(Va-wk)
    H = V.T @ Q @ V + sigma * QV.T @ QV + sigma * V.T @ Sw @ V
    rhs = QV.T @ xb + sigma * QV.T @ g0 + sigma * V.T @ Sw @ wk
    a = np.linalg.solve(H, rhs)
    return V @ a


def alg2_run(qp, sigma, lamA, lamQ, iters):
    """Algorithm 2 with S_y of eq. (3.4), S_w of eq. (2.8), from the origin, fixed sigma,
    Halpern weights 1/(k+2).  Returns per-iteration (ybar, Q wbar, zbar, xbar)."""
    A, Q = dense_of(qp)
    n, m = qp.n, qp.m
    y, w, z, x = np.zeros(m), np.zeros(n), np.zeros(n), np.zeros(n)
    y0, w0, z0, x0 = y.copy(), w.copy(), z.copy(), x.copy()
    out = []
    for k in range(iters):
        # Step 1: zbar = argmin_z L_sigma(y, w, z; x): for phi = delta_C this is the
        # Moreau decomposition of r = x + sigma(-Qw + A^*y - c)
        r = x + sigma * (-Q @ w + A.T @ y - qp.c)
        xb_ = prox_box(r, qp.L, qp.U)
        zb = (xb_ - r) / sigma
        # Step 2
        xb = x + sigma * (-Q @ w + A.T @ y + zb - qp.c)
        # Step 3-1
        wh = alg2_w_update(A, Q, qp.c, sigma, lamQ, y, zb, xb, w)
        # Step 3-2: argmin_y L_sigma(y, wh, zb; xb) + sigma/2||y - y^k||^2_{S_y}, S_y = lamA I - AA^*
        #   = argmin delta*_K(-y) + <xb, A^*y> + sigma/2||A^*y + g||^2 + sigma/2 (y-yk)'S_y(y-yk)
        #   with g = -Q wh + zb - c; the quadratic part is sigma lamA/2 ||y - v||^2 with
        #   v = y^k - (A xb + sigma A(g + A^* y^k)) / (sigma lamA), and
        #   delta*_K(-y) is the support function of -K, whose conjugate is the indicator of
        #   -K, so by Moreau  argmin delta*_K(-y) + t/2||y - v||^2 = v - Pi_{-K}(t v)/t
        #   = v + Pi_K(-t v)/t   (t = sigma lamA)
        g = -Q @ wh + zb - qp.c
        t = sigma * lamA
        v = y - (A @ xb + sigma * A @ (g + A.T @ y)) / t
        yb = v + np.minimum(np.maximum(-t * v, qp.l), qp.u) / t
        # Step 3-3
        wb = alg2_w_update(A, Q, qp.c, sigma, lamQ, yb, zb, xb, w)
        out.append((yb.copy(), Q @ wb, zb.copy(), xb.copy()))
        a, b = 1.0 / (k + 2), (k + 1.0) / (k + 2)
        y = a * y0 + b * (2 * yb - y)
        w = a * w0 + b * (2 * wb - w)
        z = a * z0 + b * (2 * zb - z)
        x = a * x0 + b * (2 * xb - x)
    return out
