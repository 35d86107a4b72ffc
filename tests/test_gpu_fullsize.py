"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

Sizes: the n = 1e6, m = 5e5 CQP (band + factor Q) and the p = 5e4 x q = 5e5 Lasso of the
benchmark configurations, and one member (c and u perturbed) of the parametric family of the
learned warm start, n = 1e5, m = 5e4.  Both sides use the same lambda_A, lambda_Q (a short oracle power
method: the trajectory only needs the two to agree on it).  Checked, normwise and element by
element:
  * the bar iterates of the first 50 steps (1, 10, 11, 20, 21, 50: R~ tests and restarts at
    multiples of 10 are crossed) to 1e-10, through the dynamic graph;
  * the bar iterate after 100 steps, one whole launch of the fixed-schedule graph with its
    fused passes, to 1e-10;
  * the converged solve: the objective to 1e-6 relative at rel-KKT <= 1e-8, with eta recomputed
    by the oracle on the GPU's output, and the iteration counts (tested every 100 steps).
The oracle needs about a minute (CQP) and two (Lasso) on one host core for the converged solve.
"""
import numpy as np
import pytest

import oracle
import qpgen
from tests.parity import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


_CACHE = {}


def _problem(name):
    if name not in _CACHE:
        if name == "large_cqp":
            qp = qpgen.large_cqp(n=1_000_000, m=500_000, seed=0)
        elif name == "lasso":
            qp = qpgen.lasso()
        else:
            qp = qpgen.param_family_instance(qpgen.param_family_base(n=100_000, m=50_000, seed=0), 7)
        lamA = oracle.power_A(qp, 50, 1e-6, 1.01) if qp.m else 0.0
        lamQ = oracle.power_Q(qp, 50, 1e-6, 1.01)
        _CACHE[name] = (qp, lamA, lamQ)
    return _CACHE[name]


@pytest.mark.parametrize("name", ["large_cqp", "lasso", "family_member"])
def test_fullsize_first_iterates(pkg, name):
    qp, lamA, lamQ = _problem(name)
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K, lambda_A=lamA, lambda_Q=lamQ)
    with pkg.Solver(qp, lambda_A=lamA, lambda_Q=lamQ) as s:
        for k in (1, 10, 11, 20, 21, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, z, w, kkt = s.get()
            # a solve capped at k steps stops at step k's stopping test, before its restart decision
            assert kkt["restarts"] == int(ref.trace["restart"][:k - 1].sum()), (name, k)
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, (name, k)
            assert close(w, ref.trace["w"][k - 1]) <= 1e-10, (name, k)
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= 1e-10, (name, k)


@pytest.mark.parametrize("name", ["large_cqp", "lasso", "family_member"])
def test_fullsize_fixed_schedule_launch(pkg, name):
    qp, lamA, lamQ = _problem(name)
    ref = oracle.solve(qp, tol=1e-30, max_iter=100, lambda_A=lamA, lambda_Q=lamQ)
    with pkg.Solver(qp, lambda_A=lamA, lambda_Q=lamQ) as s:
        s.solve(tol=1e-30, max_iter=100)
        x, y, z, w, kkt = s.get()
    assert kkt["iters"] == 100 and kkt["restarts"] == ref.restarts
    assert close(x, ref.x) <= 1e-10
    assert close(w, ref.w) <= 1e-10
    if qp.m:
        assert close(y, ref.y) <= 1e-10


@pytest.mark.parametrize("name", ["large_cqp", "lasso", "family_member"])
def test_fullsize_converged_objective(pkg, name):
    qp, lamA, lamQ = _problem(name)
    ref = oracle.solve(qp, tol=1e-8, max_iter=20000, lambda_A=lamA, lambda_Q=lamQ)
    assert ref.status == "converged"
    with pkg.Solver(qp, lambda_A=lamA, lambda_Q=lamQ) as s:
        assert s.solve(tol=1e-8, max_iter=20000) == "converged"
        x, y, z, w, kkt = s.get()
    assert abs(kkt["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj)), (kkt["pobj"], ref.pobj)
    assert abs(kkt["iters"] - ref.iters) <= 100, (kkt["iters"], ref.iters)
    e, pobj, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.05e-8, e
    assert abs(pobj - kkt["pobj"]) <= 1e-9 * (1 + abs(pobj))
