"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle runs the first iterations of the same solve on the host (a few seconds at
n = 1e6); the CUDA library, with the same lambda_A, lambda_Q, must reproduce the bar iterate
to 1e-10 relative after each checked step.  Sizes: the n=1e6/m=5e5 CQP and the p=5e4 x
q=5e5 Lasso of the benchmark configurations.
"""
import numpy as np
import pytest

import oracle
import qpgen

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("name", ["large_cqp", "lasso"])
def test_fullsize_first_iterates(pkg, name):
    qp = qpgen.large_cqp(n=1_000_000, m=500_000, seed=0) if name == "large_cqp" else qpgen.lasso()
    K = 12
    # lambda from a short power method: the trajectory only needs both sides to agree on it
    lamA = oracle.power_A(qp, 50, 1e-6, 1.01) if qp.m else 0.0
    lamQ = oracle.power_Q(qp, 50, 1e-6, 1.01)
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K, lambda_A=lamA, lambda_Q=lamQ)
    with pkg.Solver(qp, lambda_A=lamA, lambda_Q=lamQ) as s:
        for k in (1, 4, 11, 12):
            s.solve(tol=1e-30, max_iter=k)
            x, y, z, w, kkt = s.get()
            assert rel(x, ref.trace["x"][k - 1]) <= 1e-10, (name, k)
            if qp.m:
                assert rel(y, ref.trace["y"][k - 1]) <= 1e-10, (name, k)
