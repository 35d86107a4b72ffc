"""Shared-memory-tiled factor products (factor terms B^T B of Q): the one-vector products
t = B x and u = B^T t gather from column tiles of 25,600 entries held in shared memory.

Problems with more than one tile in both directions (p = 30,000 rows, n = 60,000 columns):
the tiled path (tiled_factor = 2) must reproduce the oracle's operator and first iterates to
the parity bar, reach the oracle's objective at 1e-8, and agree with the CSR path
(tiled_factor = 0).  Sums run in another order, so agreement is to rounding, not bitwise.
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
    # S: 30,000 x 60,000 with 40 entries per row (two tiles of S^T's columns, three of S's)
    yield "cqp", qpgen.large_cqp(n=60_000, m=30_000, seed=3, s_rows=30_000, s_per_row=40)
    yield "lasso", qpgen.lasso(p=30_000, q=60_000, density=5e-4, seed=2)


PROBLEMS = dict(problems())


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_tiled_operator_and_first_iterates(pkg, name):
    qp = PROBLEMS[name]
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    lam = dict(lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q)
    with pkg.Solver(qp, tiled_factor=2, **lam) as s:
        v = np.random.default_rng(0).standard_normal(qp.n)
        assert rel(s.apply("Q", v), oracle.qmul(qp, v)) <= 1e-13
        for k in (1, 2, 11, 21, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, (name, k)
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= 1e-10, (name, k)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_tiled_converges_like_the_csr_path_and_the_oracle(pkg, name):
    qp = PROBLEMS[name]
    ref = oracle.solve(qp, tol=1e-8, max_iter=100000)
    assert ref.status == "converged"
    for tiled in (2, 0):
        with pkg.Solver(qp, tiled_factor=tiled) as s:
            assert s.solve(tol=1e-8, max_iter=100000) == "converged"
            x, y, z, w, k = s.get()
        # the power method runs through the same products
        assert k["lambda_Q"] == pytest.approx(ref.lambda_Q, rel=1e-6), tiled
        assert abs(k["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj)), tiled
        e, _, _ = oracle.eta(qp, x, y, z)
        assert np.max(e) <= 1.05e-8, (tiled, e)


def test_tiled_is_chosen_for_large_factors_only(pkg):
    """The default (tiled_factor = 1) tiles a Lasso factor of 3.6e6 entries but not the factor
    of the n = 6e4 CQP (1.2e6 entries, below the 2e6 threshold)."""
    big = qpgen.lasso(p=30_000, q=60_000, density=2e-3, seed=1)   # 3.6e6 entries, 60 per column
    small = PROBLEMS["cqp"]
    with pkg.Solver(big) as s1, pkg.Solver(big, tiled_factor=0) as s0:
        v = np.random.default_rng(1).standard_normal(big.n)
        assert rel(s1.apply("Q", v), s0.apply("Q", v)) <= 1e-13
        s1.solve(tol=1e-30, max_iter=1)
        s0.solve(tol=1e-30, max_iter=1)
        assert s1.kkt()["tiled_terms"] == 1 and s0.kkt()["tiled_terms"] == 0
    with pkg.Solver(small) as s:
        v = np.random.default_rng(2).standard_normal(small.n)
        assert rel(s.apply("Q", v), oracle.qmul(small, v)) <= 1e-13
        s.solve(tol=1e-30, max_iter=1)
        assert s.kkt()["tiled_terms"] == 0
