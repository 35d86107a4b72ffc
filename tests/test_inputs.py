"""The seeded synthetic workloads hold the structure their recipes state (no GPU).

These inputs stand in for the paper's data sets (random CQPs, random Lasso, portfolio-style
QPs, the parametric family of the learned warm start); the checks run at the benchmark sizes:
shapes, entries per row, value distributions, bounds, feasibility of the planted point,
positive definiteness of the band term, and determinism in the seed.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen


def _A(qp):
    return sp.csr_matrix((qp.A_vals, qp.A_colidx, qp.A_rowptr), shape=(qp.m, qp.n))


def _csr_ok(rowptr, colidx, nrows, ncols):
    assert rowptr.dtype == np.int32 and colidx.dtype == np.int32
    assert rowptr.size == nrows + 1 and rowptr[0] == 0 and np.all(np.diff(rowptr) >= 0)
    assert colidx.size == rowptr[-1]
    assert colidx.size == 0 or (colidx.min() >= 0 and colidx.max() < ncols)
    # strictly increasing columns inside every row (distinct, sorted)
    d = np.diff(colidx.astype(np.int64))
    starts = rowptr[1:-1]
    inside = np.ones(d.size, bool)
    inside[starts[(starts > 0) & (starts < colidx.size)] - 1] = False
    assert np.all(d[inside] > 0)


@pytest.fixture(scope="module")
def cqp_1e6():
    return qpgen.large_cqp()


def test_large_cqp_recipe(cqp_1e6):
    """n = 1e6, m = 5e5; A: 6 distinct uniform columns per row, N(0,1); Q = P + S^T S with P
    symmetric pentadiagonal (diagonal U(1,2), bands U(-0.2,0.2)) and S 1e4 x n at 3 per row;
    30 % equality rows, the rest l = -inf, u = A x0 + U(0,1); C = [-5,5]^n."""
    qp = cqp_1e6
    n, m = qp.n, qp.m
    assert (n, m) == (1_000_000, 500_000)
    _csr_ok(qp.A_rowptr, qp.A_colidx, m, n)
    assert np.all(np.diff(qp.A_rowptr) == 6)
    v = qp.A_vals
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1) < 0.01
    # columns uniform: column counts have mean 3 and the Poisson-like spread of 3e6 draws
    cnt = np.bincount(qp.A_colidx, minlength=n)
    assert cnt.mean() == pytest.approx(3.0) and abs(cnt.var() - 3.0) < 0.1
    eq = qp.l == qp.u
    assert eq.sum() == 150_000 and np.all(eq[:150_000])
    assert np.all(np.isneginf(qp.l[~eq])) and np.all(np.isfinite(qp.u))
    assert np.all(qp.L == -5.0) and np.all(qp.U == 5.0)
    kinds = [t.kind for t in qp.qterms]
    assert kinds == ["dia", "factor"]
    P, S = qp.qterms
    assert list(P.offsets) == [0, 1, 2]
    assert P.diags[0].min() >= 1.0 and P.diags[0].max() < 2.0
    assert np.abs(P.diags[1:]).max() <= 0.2
    # Gershgorin: the band term is positive definite (diagonal exceeds the off-diagonal row sums)
    off = np.zeros(n)
    for k, o in ((1, 1), (2, 2)):
        a = np.abs(P.diags[k][: n - o])
        off[: n - o] += a
        off[o:] += a
    assert np.all(P.diags[0] - off > 0.19)
    assert S.p == 10_000
    _csr_ok(S.rowptr, S.colidx, S.p, n)
    assert np.all(np.diff(S.rowptr) == 3)


def test_large_cqp_planted_point_is_feasible():
    """Some x0 in U(0,1)^n (inside C) satisfies every row: rows of l = u hold A x0 exactly,
    one-sided rows with a margin in (0, 1).  Regenerated with the same stream to recover x0."""
    qp = qpgen.large_cqp(n=20_000, m=10_000, seed=4)
    rng = np.random.default_rng(4)
    qpgen.csr_k_per_row(rng, qp.m, qp.n, 6)
    qpgen.pentadiag_terms(rng, qp.n)
    qpgen.csr_k_per_row(rng, qp.qterms[1].p, qp.n, 3)
    rng.standard_normal(qp.n)
    x0 = rng.random(qp.n)
    Ax0 = _A(qp) @ x0
    eq = qp.l == qp.u
    assert np.array_equal(qp.l[eq], Ax0[eq])
    gap = qp.u[~eq] - Ax0[~eq]
    assert gap.min() >= 0 and gap.max() < 1 and abs(gap.mean() - 0.5) < 0.02


def test_plain_cqp_recipe():
    """n = 1000, m = 500; A Bernoulli(1 %), Q = M^T M with M 100 x 1000 Bernoulli(2 %);
    rows 0..249 equalities, rows 250..499 l = -inf; C = [0, 10]^n."""
    qp = qpgen.plain_cqp()
    assert (qp.n, qp.m) == (1000, 500)
    _csr_ok(qp.A_rowptr, qp.A_colidx, 500, 1000)
    assert qp.A_nnz == pytest.approx(5000, rel=0.06)
    (M,) = qp.qterms
    assert M.kind == "factor" and M.p == 100
    _csr_ok(M.rowptr, M.colidx, 100, 1000)
    assert M.colidx.size == pytest.approx(2000, rel=0.1)
    assert np.all(qp.l[:250] == qp.u[:250]) and np.all(np.isneginf(qp.l[250:]))
    assert np.all(qp.L == 0.0) and np.all(qp.U == 10.0)


def test_lasso_recipe():
    """B 5e4 x 5e5 Bernoulli(5e-4) with N(0, 1/sqrt(5e4)) values; Q = B^T B as a factor term,
    c = -B^T b, phi = lambda ||.||_1 with lambda = 0.1 ||B^T b||_inf, no rows, C = R^n."""
    qp = qpgen.lasso()
    assert (qp.n, qp.m) == (500_000, 0) and qp.phi == qpgen.PHI_L1
    (B,) = qp.qterms
    assert B.kind == "factor" and B.p == 50_000
    _csr_ok(B.rowptr, B.colidx, B.p, qp.n)
    nnz = B.colidx.size
    assert abs(nnz - 1.25e7) < 5 * np.sqrt(1.25e7)
    assert abs(B.vals.std() * np.sqrt(5e4) - 1) < 0.01
    assert qp.lam == pytest.approx(0.1 * np.abs(qp.c).max(), rel=1e-15)
    assert np.all(np.isinf(qp.L)) and np.all(np.isinf(qp.U))


@pytest.mark.parametrize("seed", [0, 1, 4095])
def test_portfolio_recipe(seed):
    """n in [50, 5000], k = max(5, n // 20) dense factor rows N(0, 1/sqrt n), diagonal
    U(0.01, 0.1); row 0 is 1^T x = 1, rows 1..10 sector sums <= 0.3 over nonempty sectors
    that partition the assets; C = [0, 0.1]^n (so 1^T x = 1 needs n >= 10)."""
    qp = qpgen.portfolio(seed)
    n = qp.n
    assert 50 <= n <= 5000 and qp.m == 11
    F, d = qp.qterms
    assert F.kind == "dense_factor" and F.p == max(5, n // 20)
    assert np.asarray(F.dense).shape == (F.p, n)
    assert d.kind == "diag" and d.dense.min() >= 0.01 and d.dense.max() < 0.1
    _csr_ok(qp.A_rowptr, qp.A_colidx, 11, n)
    A = _A(qp).toarray()
    assert np.all(A[0] == 1.0)
    assert np.all(A[1:].sum(axis=0) == 1.0) and np.all(A[1:].sum(axis=1) >= n // 10)
    assert qp.l[0] == qp.u[0] == 1.0 and np.all(np.isneginf(qp.l[1:])) and np.all(qp.u[1:] == 0.3)
    assert np.all(qp.L == 0.0) and np.all(qp.U == 0.1)


def test_parametric_family_members():
    """Members share A, Q, l, C with the base; c moves by 0.1 N(0,1); u moves by 0.1 U(0,1) on
    inequality rows only; distinct seeds give distinct members, equal seeds equal ones."""
    base = qpgen.param_family_base(n=20_000, m=10_000)
    a, a2, b = (qpgen.param_family_instance(base, s) for s in (3, 3, 4))
    assert a.qterms is base.qterms and a.A_vals is base.A_vals
    assert np.array_equal(a.l, base.l) and np.array_equal(a.L, base.L)
    eq = base.l == base.u
    assert np.array_equal(a.u[eq], base.u[eq])
    du = a.u[~eq] - base.u[~eq]
    assert du.min() >= 0 and du.max() < 0.1 and abs(du.mean() - 0.05) < 0.005
    dc = a.c - base.c
    assert abs(dc.std() - 0.1) < 0.005
    assert np.array_equal(a.c, a2.c) and np.array_equal(a.u, a2.u)
    assert not np.array_equal(a.c, b.c)
    C, U = qpgen.ws_family_data(base, [3, 4])
    assert np.array_equal(C[0], a.c) and np.array_equal(U[1], b.u)


def test_generators_are_deterministic_in_the_seed():
    for make in (lambda s: qpgen.large_cqp(n=5000, m=2500, seed=s),
                 lambda s: qpgen.lasso(p=500, q=5000, density=0.01, seed=s),
                 lambda s: qpgen.plain_cqp(seed=s),
                 lambda s: qpgen.portfolio(s)):
        x, y, z = make(7), make(7), make(8)
        for f in ("A_rowptr", "A_colidx", "A_vals", "c", "l", "u"):
            assert np.array_equal(getattr(x, f), getattr(y, f)), f
        for tx, ty in zip(x.qterms, y.qterms):
            for f in ("rowptr", "colidx", "vals", "diags", "dense"):
                if getattr(tx, f) is not None:
                    assert np.array_equal(getattr(tx, f), getattr(ty, f)), f
        assert not np.array_equal(x.c, z.c)
