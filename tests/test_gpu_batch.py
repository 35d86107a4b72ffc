"""Parity of the batched persistent solver (hprqp_batch_*) with the CPU oracle.

The batched solver runs every instance unpreconditioned, so its references run with
scaling=0 (the Sec. 4.1 preconditioning would apply to the explicit-Q instance).

Every instance of a batch runs Algorithm 4 with its own sigma, restart and termination state
inside one launch; each must reproduce the oracle's iterates (1e-10 relative at the checked
steps, same lambda_A, lambda_Q) and its converged objective (1e-6 relative at rel-KKT 1e-8).
"""
import numpy as np
import pytest

import oracle
import qpgen
from tests.parity import close  # noqa: E402

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def mixed_batch():
    # portfolio instances at both ends of the configured U{50..5000} (n = 5000: F is 250 x 5000)
    probs = [qpgen.portfolio(s, n=n) for s, n in ((1, 50), (2, 130), (3, 700), (4, 1500), (5, 61), (6, 5000))]
    probs.append(qpgen.random_small(n=40, m=12, seed=8, q_kind="csr", density=0.3))
    probs.append(qpgen.random_small(n=30, m=6, seed=9, q_kind="dense_factor", q_rank=7, phi="l1_box", lam=0.2))
    return probs


@pytest.mark.parametrize("autotune", [1, 0])
def test_batch_first_iterates(pkg, autotune):
    """autotune = 0 runs the fixed schedule, which gives the four buckets of this batch (n >= 3000,
    1500..2999, 600..1499, below 600) blocks of 512, 256, 128 and 64 threads: every block size
    reproduces the oracle's iterates."""
    probs = mixed_batch()
    K = 40
    refs = [oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K, scaling=0) for qp in probs]
    lamA = [r.lambda_A for r in refs]
    lamQ = [r.lambda_Q for r in refs]
    for k in (1, 2, 11, 21, 40):
        with pkg.BatchSolver(probs, lambda_A=lamA, lambda_Q=lamQ, autotune=autotune) as b:
            b.solve(tol=1e-30, max_iter=k)
            for i, (qp, ref) in enumerate(zip(probs, refs)):
                x, y, z, kkt = b.get(i)
                assert kkt["iters"] == k, (i, kkt)
                assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL, (i, k)
                if qp.m:
                    assert close(y, ref.trace["y"][k - 1]) <= ITER_TOL, (i, k)


def test_batch_converged(pkg):
    probs = mixed_batch()
    refs = [oracle.solve(qp, tol=1e-8, max_iter=400000, scaling=0) for qp in probs]
    with pkg.BatchSolver(probs, lambda_A=[r.lambda_A for r in refs], lambda_Q=[r.lambda_Q for r in refs]) as b:
        assert b.solve(tol=1e-8, max_iter=400000) == "converged"
        for i, (qp, ref) in enumerate(zip(probs, refs)):
            x, y, z, kkt = b.get(i)
            assert kkt["status"] == "converged"
            assert abs(kkt["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj)), i
            e, _, _ = oracle.eta(qp, x, y, z)
            assert np.max(e) <= 1.05e-8, (i, e)


def test_batch_schedule_is_reported(pkg):
    """The autotuner's choice per bucket of n (threads per instance, F in shared memory): every
    bucket with instances gets a block of 64..512 threads, an F copy only where it fits."""
    probs = mixed_batch()
    with pkg.BatchSolver(probs) as b:
        assert b.solve(tol=1e-8, max_iter=400000) == "converged"
        sched = b.schedule()
    assert [s["n_from"] for s in sched] == [3000, 1500, 600, 0]
    assert sum(s["instances"] for s in sched) == len(probs)
    assert [s["instances"] for s in sched] == [1, 1, 1, 5]
    for s in sched:
        assert s["threads"] in (64, 128, 256, 512)
        assert s["f_capacity"] >= 0 and s["f_in_smem"] == (s["f_capacity"] > 0)
    # the F copy of the largest instance (5000 x 250 doubles, 10 MB) cannot fit
    assert not sched[0]["f_in_smem"]


def test_batch_power_method_and_defaults(pkg):
    # lambda estimated inside the batch kernel (Sec. 4.1 power method): objective still agrees
    probs = [qpgen.portfolio(s, n=n) for s, n in ((11, 200), (12, 90))]
    with pkg.BatchSolver(probs) as b:
        assert b.solve(tol=1e-8, max_iter=400000) == "converged"
        for i, qp in enumerate(probs):
            ref = oracle.solve(qp, tol=1e-8, max_iter=400000, scaling=0)
            x, y, z, kkt = b.get(i)
            assert abs(kkt["lambda_Q"] - ref.lambda_Q) <= 1e-5 * ref.lambda_Q
            assert abs(kkt["lambda_A"] - ref.lambda_A) <= 1e-5 * ref.lambda_A
            assert abs(kkt["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))


def test_batch_matches_single_instance_solver(pkg):
    probs = [qpgen.portfolio(s, n=n) for s, n in ((21, 300), (22, 800))]
    with pkg.BatchSolver(probs) as b:
        b.solve(tol=1e-8)
        outs = [b.get(i) for i in range(len(probs))]
    for qp, (x, y, z, kkt) in zip(probs, outs):
        with pkg.Solver(qp, scaling=0) as s:
            s.solve(tol=1e-8)
            x1, y1, z1, w1, k1 = s.get()
        assert abs(kkt["pobj"] - k1["pobj"]) <= 1e-6 * (1 + abs(k1["pobj"]))


def test_batch_rejects_bad_input(pkg):
    qp = qpgen.random_small(n=50, m=40, seed=1)   # m above the batched limit of 32
    with pytest.raises(pkg.HPRQPError) as e:
        pkg.BatchSolver([qp])
    assert e.value.status == 4
    bad = qpgen.portfolio(1, n=60)
    bad = qpgen.QP(**{**bad.__dict__, "l": bad.u + 1.0})
    with pytest.raises(pkg.HPRQPError):
        pkg.BatchSolver([bad])
    # an empty box side: L = U = +inf on one coordinate (L in R u {-inf}, Sec. 1)
    ok = qpgen.portfolio(2, n=60)
    L, U = ok.L.copy(), ok.U.copy()
    L[5] = U[5] = np.inf
    with pytest.raises(pkg.HPRQPError) as e:
        pkg.BatchSolver([ok, qpgen.QP(**{**ok.__dict__, "L": L, "U": U})])
    assert e.value.status == 4
