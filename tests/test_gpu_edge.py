"""Edge cases of the CUDA path against the oracle.

Free rows (l = -inf, u = +inf, whose multipliers stay 0), free variables under the box
indicator, more rows than columns, a ragged size (n = 257: one 256-row chunk and one row) with
a single row, lam = 0 for the l1 term, and lam|x| plus a box with infinite sides (the dual
value phi*(-zbar) on an unbounded side).  First iterates to 1e-10 relative, the converged
objective to 1e-6 with the stopping rule recomputed by the oracle, and one separable problem
with a closed-form solution (a nonnegative l1 term among others).  Also the run-time controls:
a time-limit stop (zbar formed at hprqp_get), hprqp_profile, and the dynamic graph's chunk
length (iters_per_launch).
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
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, (name, k)
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= 1e-10, (name, k)


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


def _plain():
    return qpgen.plain_cqp(n=300, m=150, seed=3, q_rows=30, a_density=0.05, q_density=0.1)


def test_time_limit_stops_between_launches_with_a_consistent_zbar(pkg):
    """time_limit stops the solve after the launch in which it expires; hprqp_get then forms
    zbar = (xbar - r_z)/sigma from the stored iterate.  With restarts off and sigma fixed the
    run is compared with the oracle's run of the same length."""
    qp = _plain()
    lam = oracle.solve(qp, tol=1e-30, max_iter=1)
    kw = dict(restart_off=1, sigma_fixed=1)
    with pkg.Solver(qp, lambda_A=lam.lambda_A, lambda_Q=lam.lambda_Q, time_limit=0.02, **kw) as s:
        assert s.solve(tol=1e-30, max_iter=10**8) == "time_limit"
        x, y, z, w, k = s.get()
    it = k["iters"]
    assert 0 < it < 10**8 and k["status"] == "time_limit"
    ref = oracle.solve(qp, tol=1e-30, max_iter=it, lambda_A=lam.lambda_A, lambda_Q=lam.lambda_Q, **kw)
    assert close(x, ref.x) <= 1e-8 and close(y, ref.y) <= 1e-8 and close(z, ref.z) <= 1e-8, it


def test_profile_reports_every_step_kernel_and_leaves_no_solution(pkg):
    qp = _plain()
    with pkg.Solver(qp) as s:
        with pytest.raises(pkg.HPRQPError):
            s.profile(iters=5)                       # needs a solve first
        s.solve(tol=1e-30, max_iter=1)
        prof = s.profile(iters=12)
        for kind in ("zx", "pre1", "q1", "a1", "at", "pre2", "q2"):
            assert 0.0 < prof[kind] < 100.0, (kind, prof)
        with pytest.raises(pkg.HPRQPError):
            s.get()                                  # the iterate no longer belongs to a solve
        assert s.solve(tol=1e-8) == "converged"


@pytest.mark.parametrize("per", [1, 7])
def test_iters_per_launch_changes_nothing(pkg, per):
    """The dynamic graph in chunks of 1 or 7 steps runs the same kernels in the same order as in
    chunks of 64: identical iterates (fixed schedules: autotune = 0)."""
    qp = _plain()
    out = {}
    for p in (per, 64):
        with pkg.Solver(qp, autotune=0, fixed_schedule=0, iters_per_launch=p) as s:
            s.solve(tol=1e-30, max_iter=50)
            x50, y50, *_ = s.get()
            assert s.solve(tol=1e-8) == "converged"
            x, y, z, w, k = s.get()
            out[p] = (x50, y50, x, y, k["iters"])
    a, b = out[per], out[64]
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    assert a[4] == b[4]


def test_persistent_barrier_wait_gives_up_and_the_handle_recovers(pkg):
    """launch_mode 3 with a grid-barrier wait of one poll: a block that reaches a barrier before
    the others gives up at once, sets the error flag, and every block leaves at its next barrier
    (all waits bounded), so the solve returns HPRQP_TIMEOUT with the context intact.  With the
    default wait the same handle then solves to the oracle's objective."""
    qp = qpgen.large_cqp(n=5000, m=2500, seed=1)
    ref = oracle.solve(qp, tol=1e-8, max_iter=200000)
    with pkg.Solver(qp, launch_mode=3, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        s.set_wait_polls(1)
        with pytest.raises(pkg.HPRQPError) as e:
            s.solve(tol=1e-8, max_iter=200000)
        assert e.value.status == 6          # HPRQP_TIMEOUT
        s.set_wait_polls(0)
        assert s.solve(tol=1e-8, max_iter=200000) == "converged"
        k = s.kkt()
    assert abs(k["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))
