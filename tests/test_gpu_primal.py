"""Parity of the primal HPR methods of Appendix A (Algorithms 6 and 7) with the oracle.

These are ablation baselines for HPR-QP: fixed sigma, no restart, the Halpern step of Step 5.
The GPU runs their elementwise steps in its own kernels and the products A x, A^T w, Q x on
the solver's operator kernels; the iterates must match the oracle's to 1e-10 relative, and a
tolerance run must stop at the oracle's iteration with the same stopping-rule values.
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


def problems():
    yield "1d", qpgen.from_dense(np.array([[2.0]]), np.array([-4.0]), A=np.array([[1.0]]), l=np.array([-np.inf]),
                                 u=np.array([1.0]), L=np.array([-5.0]), U=np.array([5.0]))
    yield "plain", qpgen.plain_cqp(n=300, m=150, seed=3, q_rows=30, a_density=0.05, q_density=0.1)
    yield "csrQ", qpgen.random_small(n=40, m=20, seed=4, q_kind="csr", density=0.3)
    yield "l1box", qpgen.random_small(n=30, m=10, seed=6, q_kind="factor", q_rank=10, phi="l1_box", lam=0.3)
    yield "lasso", qpgen.lasso(p=400, q=2000, density=0.02)
    yield "lp", qpgen.from_dense(None, np.random.default_rng(1).standard_normal(50),
                                 A=np.random.default_rng(2).standard_normal((20, 50)),
                                 l=np.full(20, -1.0), u=np.full(20, 1.0), L=np.zeros(50), U=np.ones(50))


PROBLEMS = dict(problems())


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_primal_iterates_match_oracle(pkg, name, method):
    qp = PROBLEMS[name]
    K = 100
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K, method=method, scaling=0)
    lam = dict(lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q)
    with pkg.Solver(qp, method=method, scaling=0, **lam) as s:
        for k in (1, 2, 10, 100):
            s.solve(tol=1e-30, max_iter=k)
            x, y, z, w, kkt = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, k
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= 1e-10, k
        assert kkt["sigma"] == pytest.approx(ref.sigma, rel=1e-14)


@pytest.mark.parametrize("method", [1, 2])
def test_primal_tolerance_run_matches_oracle(pkg, method):
    qp = PROBLEMS["1d"]
    ref = oracle.solve(qp, tol=1e-4, max_iter=200000, method=method, scaling=0)
    assert ref.status == "converged"
    with pkg.Solver(qp, method=method, scaling=0, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        assert s.solve(tol=1e-4, max_iter=200000) == "converged"
        x, y, z, w, k = s.get()
    assert k["iters"] == ref.iters
    assert k["iters_1e4"] == ref.iters_1e4
    assert abs(k["pobj"] - ref.pobj) <= 1e-9 * (1 + abs(ref.pobj))
    e, _, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.01e-4


def test_primal_rejects_preconditioned_handle(pkg):
    from paper_2507_02470_gb300 import HPRQPError
    qp = PROBLEMS["csrQ"]
    with pkg.Solver(qp, method=1) as s:   # scaling=1 applies to this explicit Q
        with pytest.raises(HPRQPError):
            s.solve(tol=1e-4, max_iter=10)
