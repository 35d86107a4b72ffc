"""Parity of the preconditioned solve (Sec. 4.1: Ruiz + Pock-Chambolle) with the oracle.

The GPU and the oracle each compute the scaling, run Algorithm 4 on the scaled problem and
report the iterates in the original variables; the first iterates must agree to 1e-10, the
converged objective to 1e-6, and the stopping test must hold for the original problem.
"""
import numpy as np
import pytest

import oracle
import qpgen
from tests.parity import close  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


def stretched(seed, n=60, m=30):
    """An explicit-Q CQP whose columns of A span four orders of magnitude."""
    qp = qpgen.random_small(n=n, m=m, seed=seed, q_kind="csr", box=(-1.0, 1.0), density=0.3)
    rng = np.random.default_rng(seed)
    col = 10.0 ** rng.uniform(-2, 2, qp.n)
    qp.A_vals = qp.A_vals * col[qp.A_colidx]
    return qp


@pytest.mark.parametrize("seed", [69, 70])
def test_scaled_first_iterates_and_objective(pkg, seed):
    qp = stretched(seed)
    K = 30
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        for k in (1, 2, 10, 11, 30):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, k
            assert close(y, ref.trace["y"][k - 1]) <= 1e-10, k
    full = oracle.solve(qp, tol=1e-8, max_iter=400000)
    assert full.status == "converged"
    with pkg.Solver(qp, lambda_A=full.lambda_A, lambda_Q=full.lambda_Q) as s:
        assert s.solve(tol=1e-8, max_iter=400000) == "converged"
        x, y, z, w, k = s.get()
    assert abs(k["pobj"] - full.pobj) <= 1e-6 * (1 + abs(full.pobj))
    e, _, _ = oracle.eta(qp, x, y, z)          # the original problem's stopping rule
    assert np.max(e) <= 1.05e-8, e
    assert np.all(x >= qp.L - 1e-12) and np.all(x <= qp.U + 1e-12)


def test_scaling_off_agrees_and_needs_more_iterations(pkg):
    qp = stretched(69)
    with pkg.Solver(qp) as s:
        assert s.solve(tol=1e-8, max_iter=400000) == "converged"
        on = s.kkt()
    with pkg.Solver(qp, scaling=0) as s:
        assert s.solve(tol=1e-8, max_iter=400000) == "converged"
        off = s.kkt()
    assert abs(on["pobj"] - off["pobj"]) <= 1e-6 * (1 + abs(off["pobj"]))
    assert on["iters"] < off["iters"]


def test_scaled_apply_warm_start_and_set_data(pkg):
    qp = stretched(70)
    from tests import dense_ref as D
    A, Q = D.dense_of(qp)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(qp.n)
    u = rng.standard_normal(qp.m)
    x0 = np.clip(rng.standard_normal(qp.n) * 0.3, qp.L, qp.U)
    y0 = rng.standard_normal(qp.m) * 0.1
    with pkg.Solver(qp) as s:
        # operators in the original variables
        assert np.allclose(s.apply("A", v), A @ v, rtol=1e-12, atol=1e-12 * np.abs(A).max())
        assert np.allclose(s.apply("AT", u), A.T @ u, rtol=1e-12, atol=1e-12 * np.abs(A).max())
        assert np.allclose(s.apply("Q", v), Q @ v, rtol=1e-12, atol=1e-12 * np.abs(Q).max())
        # warm start given in the original variables
        ref = oracle.solve(qp, tol=1e-30, max_iter=15, x0=x0, y0=y0, trace_len=15)
        s.set_lambda(ref.lambda_A, ref.lambda_Q)
        s.set_warm_start(x0, y0)
        s.solve(tol=1e-30, max_iter=15)
        x, y, *_ = s.get()
        assert close(x, ref.trace["x"][14]) <= 1e-10 and close(y, ref.trace["y"][14]) <= 1e-10
        # new c: the stored (scaled) data are replaced consistently
        s.set_warm_start(None, None)
        c2 = qp.c + 0.3 * rng.standard_normal(qp.n)
        s.set_data(c=c2)
        s.set_lambda(0.0, 0.0)
        assert s.solve(tol=1e-8, max_iter=400000) == "converged"
        k = s.kkt()
    qp.c = c2
    ref2 = oracle.solve(qp, tol=1e-8, max_iter=400000)
    assert abs(k["pobj"] - ref2.pobj) <= 1e-6 * (1 + abs(ref2.pobj))
