"""Edge cases of the CUDA path against the oracle.

Free rows (l = -inf, u = +inf, whose multipliers stay 0), free variables under the box
indicator, more rows than columns, a ragged size (n = 257: one 256-row chunk and one row) with
a single row, lam = 0 for the l1 term, and lam|x| plus a box with infinite sides (the dual
value phi*(-zbar) on an unbounded side).  First iterates to 1e-10 relative, the converged
objective to 1e-6 with the stopping rule recomputed by the oracle, and one separable problem
with a closed-form solution (a nonnegative l1 term among others).
"""
import numpy as np
import pytest

import oracle
import qpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


def edge_problems():
    rng = np.random.default_rng(21)
    qp = qpgen.plain_cqp(n=300, m=150, seed=8, q_rows=30, a_density=0.05, q_density=0.1)
    qp.l = qp.l.copy()
    qp.u = qp.u.copy()
    qp.l[100:120] = -np.inf
    qp.u[100:120] = np.inf
    yield "free_rows", qp
    qp = qpgen.random_small(n=60, m=25, seed=12, q_kind="csr", density=0.3, box=(-1.0, 1.0))
    qp.L = qp.L.copy()
    qp.U = qp.U.copy()
    qp.L[::3] = -np.inf
    qp.U[::3] = np.inf
    yield "free_vars", qp
    n, m = 200, 700
    A = np.where(rng.random((m, n)) < 0.05, rng.standard_normal((m, n)), 0.0)
    x0 = rng.uniform(-0.5, 0.5, n)
    Ax0 = A @ x0
    F = rng.standard_normal((40, n))
    yield "tall", qpgen.from_dense(F.T @ F / n, rng.standard_normal(n), A=A, l=Ax0 - rng.random(m),
                                   u=Ax0 + rng.random(m), L=np.full(n, -1.0), U=np.full(n, 1.0))
    n = 257
    F = rng.standard_normal((30, n))
    yield "n257_m1", qpgen.from_dense(F.T @ F / n + np.eye(n) * 0.1, rng.standard_normal(n),
                                      A=np.ones((1, n)), l=np.array([1.0]), u=np.array([1.0]),
                                      L=np.zeros(n), U=np.full(n, 0.05))
    qp = qpgen.random_small(n=40, m=15, seed=13, q_kind="csr", density=0.4, box=(-np.inf, np.inf))
    qp.phi = qpgen.PHI_L1
    qp.lam = 0.0
    yield "l1_zero", qp
    qp = qpgen.random_small(n=40, m=15, seed=14, q_kind="factor", q_rank=15, phi="l1_box", lam=0.2)
    qp.L = qp.L.copy()
    qp.U = qp.U.copy()
    qp.L[:10] = -np.inf
    qp.U[10:20] = np.inf
    yield "l1box_inf", qp


PROBLEMS = dict(edge_problems())


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_edge_first_iterates(pkg, name):
    qp = PROBLEMS[name]
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    with pkg.Solver(qp, lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q) as s:
        for k in (1, 2, 10, 11, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert rel(x, ref.trace["x"][k - 1]) <= 1e-10, (name, k)
            if qp.m:
                assert rel(y, ref.trace["y"][k - 1]) <= 1e-10, (name, k)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_edge_converged_objective(pkg, name):
    qp = PROBLEMS[name]
    ref = oracle.solve(qp, tol=1e-8, max_iter=200000)
    assert ref.status == "converged"
    with pkg.Solver(qp) as s:
        assert s.solve(tol=1e-8, max_iter=200000) == "converged"
        x, y, z, w, k = s.get()
    assert abs(k["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))
    e, _, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.05e-8, e
    if name == "free_rows":
        assert np.all(y[100:120] == 0.0)


def test_l1_with_unbounded_sides_closed_form(pkg):
    """lam|x| + [L, U] with x >= 0, x <= U and free coordinates, diagonal Q: the solution is
    clip(soft(-c, lam)/q, L, U) coordinate by coordinate."""
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = 2 * rng.standard_normal(n)
    L = np.where(np.arange(n) % 4 == 0, 0.0, -np.inf)
    U = np.where(np.arange(n) % 4 == 1, 0.4, np.inf)
    L[2::4], U[2::4] = -0.3, 0.3
    lam = 0.3
    qp = qpgen.from_dense(np.diag(q), c, L=L, U=U, phi="l1_box", lam=lam, q_kind="diag")
    with pkg.Solver(qp) as s:
        assert s.solve(tol=1e-10, max_iter=400000) == "converged"
        x, *_ = s.get()
    soft = np.sign(-c) * np.maximum(np.abs(c) - lam, 0)
    np.testing.assert_allclose(x, np.clip(soft / q, L, U), atol=1e-8)
