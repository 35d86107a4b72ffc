"""Seeded synthetic QP instances for HPR-QP (problem data only).

This module builds the problem data  min 1/2<x,Qx> + <c,x> + phi(x)  s.t.  l <= Ax <= u
(the CCQP of Sec. 1, eq. (1.1); box phi is the CQP of eq. (1.2)).  It holds none of the
solver's arithmetic: it draws random matrices and vectors and assembles CSR arrays.  Both
the CUDA library's tests and the CPU oracle consume the same objects.

Q is described as a sum of terms (``QTerm``), each one of
  * ``diag``      Q += diag(d)
  * ``csr``       Q += an explicit symmetric n x n CSR matrix
  * ``dia``       Q += a symmetric banded matrix stored by its upper diagonals
                  (offsets >= 0, diags[k][i] = Q[i, i+off_k], entries past the end are 0)
  * ``factor``    Q += B^T B with B a p x n CSR matrix (matrix-free, Sec. 1 "no explicit Q")
  * ``dense_factor``  Q += F^T F with F a dense row-major p x n matrix
An empty term list means Q = 0 (the LP special case, Sec. 2.2 remark).

Infinite bounds are IEEE +-inf.  phi is one of ``box`` (indicator of [L,U]), ``l1``
(lam*||x||_1) or ``l1_box`` (both).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

PHI_BOX, PHI_L1, PHI_L1_BOX = 0, 1, 2
_PHI_NAMES = {"box": PHI_BOX, "l1": PHI_L1, "l1_box": PHI_L1_BOX}


@dataclass
class QTerm:
    kind: str                                   # diag | csr | dia | factor | dense_factor | qap
    p: int = 0                                  # rows of B or F
    rowptr: Optional[np.ndarray] = None         # int32
    colidx: Optional[np.ndarray] = None         # int32
    vals: Optional[np.ndarray] = None           # float64
    offsets: Optional[np.ndarray] = None        # int32, dia only
    diags: Optional[np.ndarray] = None          # float64 [ndiag, n], dia only
    dense: Optional[np.ndarray] = None          # float64: diag (n,), F (p, n) row-major, or the four
                                                # symmetric d x d matrices of a qap term (p = d)


@dataclass
class QP:
    n: int
    m: int
    A_rowptr: np.ndarray
    A_colidx: np.ndarray
    A_vals: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    L: np.ndarray
    U: np.ndarray
    phi: int = PHI_BOX
    lam: float = 0.0
    qterms: List[QTerm] = field(default_factory=list)
    name: str = ""

    @property
    def A_nnz(self) -> int:
        return int(self.A_rowptr[-1]) if self.m > 0 else 0

    def A_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.A_vals, self.A_colidx, self.A_rowptr), shape=(self.m, self.n))

    def Q_scipy(self) -> sp.csr_matrix:
        """Assembled Q (for small test problems and CSR comparisons only)."""
        Q = sp.csr_matrix((self.n, self.n))
        for t in self.qterms:
            Q = Q + qterm_scipy(t, self.n)
        return sp.csr_matrix(Q)


def qterm_scipy(t: QTerm, n: int) -> sp.csr_matrix:
    if t.kind == "diag":
        return sp.diags(t.dense, 0, shape=(n, n), format="csr")
    if t.kind == "csr":
        return sp.csr_matrix((t.vals, t.colidx, t.rowptr), shape=(n, n))
    if t.kind == "dia":
        M = sp.csr_matrix((n, n))
        for k, off in enumerate(t.offsets):
            off = int(off)
            d = t.diags[k][: n - off]
            if off == 0:
                M = M + sp.diags(d, 0, shape=(n, n))
            else:
                M = M + sp.diags(d, off, shape=(n, n)) + sp.diags(d, -off, shape=(n, n))
        return sp.csr_matrix(M)
    if t.kind == "factor":
        B = sp.csr_matrix((t.vals, t.colidx, t.rowptr), shape=(t.p, n))
        return sp.csr_matrix(B.T @ B)
    if t.kind == "dense_factor":
        F = np.asarray(t.dense).reshape(t.p, n)
        return sp.csr_matrix(F.T @ F)
    if t.kind == "qap":
        d = t.p
        M = np.asarray(t.dense).reshape(4, d, d)
        I = np.eye(d)
        # column-major vec: vec(A X B) = (B^T kron A) vec(X), vec(S X) = (I kron S), vec(X T) = (T^T kron I)
        return sp.csr_matrix(np.kron(M[1], M[0]) - np.kron(I, M[2]) - np.kron(M[3], I))
    raise ValueError(t.kind)


# --------------------------------------------------------------------------------------
# construction helpers
# --------------------------------------------------------------------------------------

def csr_from_scipy(M) -> tuple:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return (M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def _rows_k_distinct(rng: np.random.Generator, nrows: int, ncols: int, k: int) -> np.ndarray:
    """nrows x k matrix of column indices, k distinct uniform columns per row, sorted."""
    cols = rng.integers(0, ncols, size=(nrows, k), dtype=np.int64)
    cols.sort(axis=1)
    while True:
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1) if k > 1 else np.zeros(nrows, bool)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            return cols
        redo = rng.integers(0, ncols, size=(bad.size, k), dtype=np.int64)
        redo.sort(axis=1)
        cols[bad] = redo


def csr_k_per_row(rng, nrows, ncols, k, scale=1.0):
    cols = _rows_k_distinct(rng, nrows, ncols, k)
    vals = rng.standard_normal((nrows, k)) * scale
    rowptr = (np.arange(nrows + 1, dtype=np.int64) * k).astype(np.int32)
    return rowptr, cols.reshape(-1).astype(np.int32), vals.reshape(-1).astype(np.float64)


def csr_bernoulli(rng, nrows, ncols, p, scale=1.0):
    """Independent Bernoulli(p) pattern per entry, N(0, scale) values."""
    counts = rng.binomial(ncols, p, size=nrows)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colidx = np.empty(nnz, dtype=np.int32)
    for i in range(nrows):
        k = int(counts[i])
        if k == 0:
            continue
        if k * 4 < ncols:
            c = np.unique(rng.integers(0, ncols, size=k + 8 + k // 8))
            while c.size < k:
                c = np.unique(np.concatenate([c, rng.integers(0, ncols, size=k)]))
            c = np.sort(rng.permutation(c)[:k])
        else:
            c = np.sort(rng.permutation(ncols)[:k])
        colidx[rowptr[i]:rowptr[i + 1]] = c
    vals = rng.standard_normal(nnz) * scale
    if nnz >= 2 ** 31:
        raise ValueError("nnz too large for int32 row pointers")
    return rowptr.astype(np.int32), colidx, vals.astype(np.float64)


def csr_bernoulli_fast(rng, nrows, ncols, p, scale=1.0):
    """Bernoulli(p) pattern for large sparse matrices, drawn row by row in bulk."""
    counts = rng.binomial(ncols, p, size=nrows).astype(np.int64)
    nnz = int(counts.sum())
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    rows = np.repeat(np.arange(nrows, dtype=np.int64), counts)
    cols = rng.integers(0, ncols, size=nnz, dtype=np.int64)
    key = rows * ncols + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    # redraw duplicates until the pattern is a set (keeps the per-row counts)
    while True:
        dup = np.nonzero(key[1:] == key[:-1])[0] + 1
        if dup.size == 0:
            break
        r = key[dup] // ncols
        key[dup] = r * ncols + rng.integers(0, ncols, size=dup.size, dtype=np.int64)
        key.sort()
    colidx = (key % ncols).astype(np.int32)
    vals = rng.standard_normal(nnz) * scale
    return rowptr.astype(np.int32), colidx, vals.astype(np.float64)


def _csr_matvec(rowptr, colidx, vals, x):
    nrows = rowptr.size - 1
    M = sp.csr_matrix((vals, colidx, rowptr), shape=(nrows, x.size))
    return M @ x


def _bounds_eq_then_upper(rng, Ax0, n_eq):
    """First n_eq rows l = u = A x0; remaining rows l = -inf, u = A x0 + U(0,1)."""
    m = Ax0.size
    l = np.full(m, -np.inf)
    u = Ax0 + rng.random(m)
    l[:n_eq] = Ax0[:n_eq]
    u[:n_eq] = Ax0[:n_eq]
    return l, u


# --------------------------------------------------------------------------------------
# the five workload families
# --------------------------------------------------------------------------------------

def plain_cqp(n=1000, m=500, seed=0, a_density=0.01, q_rows=100, q_density=0.02,
              n_eq=None, box=(0.0, 10.0)) -> QP:
    """Plain FP64 CQP: A Bernoulli(1%) N(0,1); Q = M^T M with M q_rows x n Bernoulli(2%);
    c ~ N(0,1); x0 ~ U(0,1); rows [0, m/2) equalities l=u=A x0, the rest l=-inf,
    u = A x0 + U(0,1); C = [0,10]^n."""
    rng = np.random.default_rng(seed)
    A = csr_bernoulli(rng, m, n, a_density)
    M = csr_bernoulli(rng, q_rows, n, q_density)
    c = rng.standard_normal(n)
    x0 = rng.random(n)
    Ax0 = _csr_matvec(*A, x0) if m > 0 else np.zeros(0)
    l, u = _bounds_eq_then_upper(rng, Ax0, m // 2 if n_eq is None else n_eq)
    L = np.full(n, box[0])
    U = np.full(n, box[1])
    q = QTerm("factor", p=q_rows, rowptr=M[0], colidx=M[1], vals=M[2])
    return QP(n, m, A[0], A[1], A[2], c, l, u, L, U, PHI_BOX, 0.0, [q],
              name=f"plain_cqp_n{n}_m{m}_s{seed}")


def pentadiag_terms(rng, n):
    """Symmetric pentadiagonal P: diag U(1,2), bands +-1, +-2 U(-0.2,0.2) (row sums of
    |off-diagonals| <= 0.8 < 1 <= diag, so P is positive definite)."""
    d0 = 1.0 + rng.random(n)
    d1 = rng.uniform(-0.2, 0.2, n)
    d2 = rng.uniform(-0.2, 0.2, n)
    d1[n - 1:] = 0.0
    d2[max(n - 2, 0):] = 0.0
    return QTerm("dia", offsets=np.array([0, 1, 2], np.int32), diags=np.stack([d0, d1, d2]))


def large_cqp(n=1_000_000, m=500_000, seed=0, s_rows=None, eq_frac=0.3, a_per_row=6,
              s_per_row=3, box=(-5.0, 5.0), q_as="sum") -> QP:
    """Large sparse CQP: A with 6 uniform distinct columns per row, N(0,1);
    Q = P (pentadiagonal) + S^T S with S s_rows x n, 3 nnz per row N(0,1);
    c ~ N(0,1); 30% equality rows, the rest one-sided; C = [-5,5]^n.
    ``q_as='sum'`` passes Q as dia + factor terms, ``'csr'`` as one assembled CSR."""
    rng = np.random.default_rng(seed)
    if s_rows is None:
        s_rows = max(1, n // 100)
    A = csr_k_per_row(rng, m, n, a_per_row)
    P = pentadiag_terms(rng, n)
    S = csr_k_per_row(rng, s_rows, n, s_per_row)
    c = rng.standard_normal(n)
    x0 = rng.random(n)
    Ax0 = _csr_matvec(*A, x0)
    l, u = _bounds_eq_then_upper(rng, Ax0, int(round(eq_frac * m)))
    L = np.full(n, box[0])
    U = np.full(n, box[1])
    fac = QTerm("factor", p=s_rows, rowptr=S[0], colidx=S[1], vals=S[2])
    if q_as == "sum":
        terms = [P, fac]
    else:
        Q = qterm_scipy(P, n) + qterm_scipy(fac, n)
        rp, ci, va = csr_from_scipy(Q)
        terms = [QTerm("csr", rowptr=rp, colidx=ci, vals=va)]
    return QP(n, m, A[0], A[1], A[2], c, l, u, L, U, PHI_BOX, 0.0, terms,
              name=f"large_cqp_n{n}_m{m}_s{seed}_{q_as}")


def lasso(p=50_000, q=500_000, seed=0, density=5e-4, support_frac=0.01, noise=0.01,
          lam_frac=0.1) -> QP:
    """Lasso min 1/2||Bx-b||^2 + lam||x||_1 as a CCQP (Sec. 4.4, original form):
    Q = B^T B matrix-free, c = -B^T b, phi = lam||.||_1 with lam = 0.1||B^T b||_inf,
    no A rows, C = R^n.  B is p x q Bernoulli(density), N(0, 1/sqrt(p))."""
    rng = np.random.default_rng(seed)
    B = csr_bernoulli_fast(rng, p, q, density, scale=1.0 / np.sqrt(p))
    k = max(1, int(round(support_frac * q)))
    xs = np.zeros(q)
    xs[rng.permutation(q)[:k]] = rng.standard_normal(k)
    Bm = sp.csr_matrix((B[2], B[1], B[0]), shape=(p, q))
    b = Bm @ xs + noise * rng.standard_normal(p)
    Btb = Bm.T @ b
    c = -Btb
    lam = lam_frac * float(np.max(np.abs(Btb)))
    e = np.zeros(0, np.int32)
    return QP(q, 0, np.zeros(1, np.int32), e, np.zeros(0), c, np.zeros(0), np.zeros(0),
              np.full(q, -np.inf), np.full(q, np.inf), PHI_L1, lam,
              [QTerm("factor", p=p, rowptr=B[0], colidx=B[1], vals=B[2])],
              name=f"lasso_p{p}_q{q}_s{seed}")


def portfolio(seed: int, n: Optional[int] = None, n_lo=50, n_hi=5000, sectors=10) -> QP:
    """Portfolio-style CQP: Q = F^T F + diag(U(0.01,0.1)), F k x n dense N(0, 1/sqrt(n)),
    k = max(5, n//20); A = [1^T; 10 sector indicator rows] with 1^T x = 1 and sector
    sums <= 0.3; c ~ N(0, 0.1); C = [0, 0.1]^n.  Sectors are assigned round-robin and
    then shuffled, so none is empty."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(rng.integers(n_lo, n_hi + 1))
    k = max(5, n // 20)
    F = rng.standard_normal((k, n)) / np.sqrt(n)
    d = rng.uniform(0.01, 0.1, n)
    sector = rng.permutation(np.arange(n) % sectors)
    m = 1 + sectors
    rows = [np.arange(n)] + [np.nonzero(sector == s)[0] for s in range(sectors)]
    rowptr = np.zeros(m + 1, np.int64)
    rowptr[1:] = np.cumsum([r.size for r in rows])
    colidx = np.concatenate(rows).astype(np.int32)
    vals = np.ones(colidx.size)
    l = np.concatenate([[1.0], np.full(sectors, -np.inf)])
    u = np.concatenate([[1.0], np.full(sectors, 0.3)])
    c = 0.1 * rng.standard_normal(n)
    terms = [QTerm("dense_factor", p=k, dense=np.ascontiguousarray(F)), QTerm("diag", dense=d)]
    return QP(n, m, rowptr.astype(np.int32), colidx, vals, c, l, u, np.zeros(n),
              np.full(n, 0.1), PHI_BOX, 0.0, terms, name=f"portfolio_n{n}_s{seed}")


def param_family_base(n=100_000, m=50_000, seed=0, s_rows=None):
    """The fixed part of the parametric family: A and Q of ``large_cqp`` at (n, m),
    and the nominal c-bar, u-bar."""
    base = large_cqp(n=n, m=m, seed=seed, s_rows=s_rows if s_rows is not None else max(1, n // 100))
    return base


def param_family_instance(base: QP, seed: int) -> QP:
    """One member: c = c-bar + 0.1 N(0,1), u = u-bar + 0.1 U(0,1) on inequality rows."""
    rng = np.random.default_rng(1_000_003 + seed)
    c = base.c + 0.1 * rng.standard_normal(base.n)
    u = base.u.copy()
    ineq = np.isinf(base.l)
    u[ineq] = u[ineq] + 0.1 * rng.random(int(ineq.sum()))
    return QP(base.n, base.m, base.A_rowptr, base.A_colidx, base.A_vals, c, base.l, u,
              base.L, base.U, base.phi, base.lam, base.qterms, name=f"{base.name}_i{seed}")


def ws_gaussian(rows: int, cols: int, seed: int) -> np.ndarray:
    """A rows x cols float32 matrix of independent N(0, 1) draws (seeded), the raw material
    of the fixed random projection P and decoder basis Phi of the learned warm start; the
    caller applies the scale."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((rows, cols), dtype=np.float32)


def ws_family_data(base: QP, seeds) -> tuple:
    """(c, u) of the family members with the given seeds, stacked as float64 arrays
    (len(seeds) x n and len(seeds) x m), as ``param_family_instance`` draws them."""
    seeds = list(seeds)
    C = np.empty((len(seeds), base.n))
    U = np.empty((len(seeds), base.m))
    for k, sd in enumerate(seeds):
        q = param_family_instance(base, sd)
        C[k] = q.c
        U[k] = q.u
    return C, U


def qap_matrices(d: int, seed: int = 0):
    """A QAPLIB-like pair: a symmetric flow matrix (integers 0..9 on 60 % of the pairs, zero
    diagonal) and the Manhattan distances of d random points on a sqrt(d)-sized grid."""
    rng = np.random.default_rng(seed)
    F = rng.integers(0, 10, (d, d)) * (rng.random((d, d)) < 0.6)
    F = np.triu(F, 1)
    F = (F + F.T).astype(np.float64)
    side = max(2, int(np.ceil(np.sqrt(d))) + 1)
    pts = rng.integers(0, side, (d, 2))
    D = np.abs(pts[:, None, :] - pts[None, :, :]).sum(axis=2).astype(np.float64)
    return F, D


def qap_relaxation(d: int = 16, seed: int = 0, Ahat=None, Bhat=None) -> QP:
    """The convex QAP relaxation of Sec. 4.5: min <vec X, Qhat vec X> over doubly stochastic
    X >= 0, Qhat = Bhat (x) Ahat - I (x) S - T (x) I, passed as one matrix-free "qap" term
    (Q = 2 Qhat, c = 0).  S = V_A diag(s) V_A^T, T = V_B diag(t) V_B^T from the eigen-
    decompositions of Ahat (alpha descending) and Bhat (beta ascending) and an optimal (s, t)
    of max <e, s + t> s.t. s_i + t_j <= alpha_i beta_j, solved numerically (HiGHS)."""
    import scipy.optimize as so
    if Ahat is None or Bhat is None:
        Ahat, Bhat = qap_matrices(d, seed)
    d = Ahat.shape[0]
    aw, av = np.linalg.eigh(Ahat)
    oa = np.argsort(-aw)
    alpha, VA = aw[oa], av[:, oa]
    bw, bv = np.linalg.eigh(Bhat)
    ob = np.argsort(bw)
    beta, VB = bw[ob], bv[:, ob]
    # LP in (s, t): rows s_i + t_j <= alpha_i beta_j
    ii, jj = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    rows = np.arange(d * d)
    Aub = sp.csr_matrix((np.ones(2 * d * d), (np.concatenate([rows, rows]),
                                              np.concatenate([ii.ravel(), d + jj.ravel()]))), shape=(d * d, 2 * d))
    res = so.linprog(-np.ones(2 * d), A_ub=Aub, b_ub=np.outer(alpha, beta).ravel(), bounds=(None, None),
                     method="highs")
    if res.status != 0:
        raise RuntimeError(f"QAP bound LP failed: {res.message}")
    sv, tv = res.x[:d], res.x[d:]
    S = VA @ np.diag(sv) @ VA.T
    T = VB @ np.diag(tv) @ VB.T
    S = 0.5 * (S + S.T)
    T = 0.5 * (T + T.T)
    n = d * d
    dense = np.concatenate([2.0 * Ahat, Bhat, 2.0 * S, 2.0 * T]).reshape(-1)
    term = QTerm("qap", p=d, dense=dense)
    # X e = e (row sums) and X^T e = e (column sums), vec(X)[i + j d] = X[i][j]
    r_rows = np.repeat(np.arange(d), d)                 # row-sum constraint i: entries (i, j) for all j
    r_cols = (np.arange(d)[:, None] + d * np.arange(d)[None, :]).ravel()
    c_rows = d + np.repeat(np.arange(d), d)             # column-sum constraint j: entries (i, j) for all i
    c_cols = (np.arange(d)[None, :] + d * np.arange(d)[:, None]).ravel()
    Amat = sp.csr_matrix((np.ones(2 * n), (np.concatenate([r_rows, c_rows]), np.concatenate([r_cols, c_cols]))),
                         shape=(2 * d, n))
    rp, ci, va = csr_from_scipy(Amat)
    qp = QP(n, 2 * d, rp, ci, va, np.zeros(n), np.ones(2 * d), np.ones(2 * d), np.zeros(n), np.full(n, np.inf),
            PHI_BOX, 0.0, [term], name=f"qap_d{d}_s{seed}")
    qp.qap_bound_const = float(sv.sum() + tv.sum())
    qp.qap_Ahat, qp.qap_Bhat = Ahat, Bhat
    return qp


# --------------------------------------------------------------------------------------
# small problems for tests (closed forms, brute force, special cases)
# --------------------------------------------------------------------------------------

def random_small(n=6, m=4, seed=0, q_kind="csr", q_rank=None, phi="box", lam=0.0,
                 eq_rows=1, box=(-1.0, 1.0), density=0.6) -> QP:
    """Small dense-ish random CQP used by brute-force and equivalence tests."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    for i in range(m):
        if not np.any(A[i]):
            A[i, rng.integers(n)] = 1.0
    r = n if q_rank is None else q_rank
    Fq = rng.standard_normal((r, n))
    Qd = Fq.T @ Fq if r > 0 else np.zeros((n, n))
    c = rng.standard_normal(n)
    x0 = rng.uniform(box[0] * 0.5, box[1] * 0.5, n) if np.isfinite(box[0]) else rng.standard_normal(n)
    Ax0 = A @ x0
    l = Ax0 - rng.random(m)
    u = Ax0 + rng.random(m)
    l[:eq_rows] = Ax0[:eq_rows]
    u[:eq_rows] = Ax0[:eq_rows]
    if m > eq_rows + 1:
        l[eq_rows + 1::2] = -np.inf
    rp, ci, va = csr_from_scipy(sp.csr_matrix(A))
    terms: List[QTerm] = []
    if r > 0:
        if q_kind == "csr":
            qrp, qci, qva = csr_from_scipy(sp.csr_matrix(Qd))
            terms = [QTerm("csr", rowptr=qrp, colidx=qci, vals=qva)]
        elif q_kind == "factor":
            frp, fci, fva = csr_from_scipy(sp.csr_matrix(Fq))
            terms = [QTerm("factor", p=r, rowptr=frp, colidx=fci, vals=fva)]
        elif q_kind == "dense_factor":
            terms = [QTerm("dense_factor", p=r, dense=np.ascontiguousarray(Fq))]
        else:
            raise ValueError(q_kind)
    return QP(n, m, rp, ci, va, c, l, u, np.full(n, box[0]), np.full(n, box[1]),
              _PHI_NAMES[phi], lam, terms, name=f"small_n{n}_m{m}_s{seed}_{q_kind}_{phi}")


def from_dense(Q: np.ndarray, c, A=None, l=None, u=None, L=None, U=None, phi="box",
               lam=0.0, q_kind="csr") -> QP:
    """Wrap dense test data (Q symmetric PSD) into a QP."""
    n = c.size
    A = np.zeros((0, n)) if A is None else np.asarray(A, float)
    m = A.shape[0]
    rp, ci, va = csr_from_scipy(sp.csr_matrix(A)) if m > 0 else (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    terms = []
    if Q is not None and np.any(Q):
        if q_kind == "csr":
            qrp, qci, qva = csr_from_scipy(sp.csr_matrix(Q))
            terms = [QTerm("csr", rowptr=qrp, colidx=qci, vals=qva)]
        elif q_kind == "diag":
            terms = [QTerm("diag", dense=np.diag(Q).copy())]
        else:
            raise ValueError(q_kind)
    return QP(n, m, rp, ci, va, np.asarray(c, float),
              np.zeros(0) if l is None else np.asarray(l, float),
              np.zeros(0) if u is None else np.asarray(u, float),
              np.full(n, -np.inf) if L is None else np.asarray(L, float),
              np.full(n, np.inf) if U is None else np.asarray(U, float),
              _PHI_NAMES[phi], lam, terms, name="dense")
