"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Bar: the first iterates agree to 1e-10 relative, both normwise (||a-b|| / max(1, ||b||)) and
element by element (max_i |a_i - b_i| / max(1, ||b||_inf)), the converged objective to 1e-6
relative at rel-KKT <= 1e-8, operator products to 1e-13 relative.  The
iteration trajectory depends on lambda_A, lambda_Q and sigma0 only through the data, so
the parity runs pass the oracle's power-method estimates to both sides.
"""
import numpy as np
import pytest

import oracle
import qpgen
from tests.parity import close, rel

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
OBJ_TOL = 1e-6


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def small_problems():
    yield "plain", qpgen.plain_cqp(n=300, m=150, seed=3, q_rows=30, a_density=0.05, q_density=0.1)
    yield "csrQ", qpgen.random_small(n=40, m=20, seed=4, q_kind="csr", density=0.3)
    yield "dense", qpgen.portfolio(5, n=700)
    yield "l1box", qpgen.random_small(n=30, m=10, seed=6, q_kind="factor", q_rank=10, phi="l1_box", lam=0.3)
    yield "lasso", qpgen.lasso(p=400, q=2000, density=0.02)
    yield "lp", qpgen.from_dense(None, np.random.default_rng(1).standard_normal(50),
                                 A=np.random.default_rng(2).standard_normal((20, 50)),
                                 l=np.full(20, -1.0), u=np.full(20, 1.0), L=np.zeros(50), U=np.ones(50))
    yield "large_sum", qpgen.large_cqp(n=5000, m=2500, seed=1)


PROBLEMS = dict(small_problems())


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_operators(pkg, name):
    qp = PROBLEMS[name]
    rng = np.random.default_rng(0)
    with pkg.Solver(qp) as s:
        v = rng.standard_normal(qp.n)
        assert rel(s.apply("Q", v), oracle.qmul(qp, v)) <= 1e-13
        if qp.m:
            yv = rng.standard_normal(qp.m)
            assert rel(s.apply("A", v), oracle.amul(qp, v)) <= 1e-13
            assert rel(s.apply("AT", yv), oracle.atmul(qp, yv)) <= 1e-13


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_first_iterates(pkg, name):
    qp = PROBLEMS[name]
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    lamA, lamQ = ref.lambda_A, ref.lambda_Q
    with pkg.Solver(qp, lambda_A=lamA if qp.m else 0.0, lambda_Q=lamQ) as s:
        for k in (1, 2, 3, 10, 11, 20, 21, 33, 41, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, z, w, kkt = s.get()
            assert kkt["iters"] == k
            ex = close(x, ref.trace["x"][k - 1])
            assert ex <= ITER_TOL, (name, k, ex)
            if qp.m:
                ey = close(y, ref.trace["y"][k - 1])
                assert ey <= ITER_TOL, (name, k, ey)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_iterates_through_the_fixed_schedule_graph(pkg, name):
    """Whole periods of 100 steps run through the fixed-schedule graph, whose plain steps end
    with the fused passes (A^T ybar with the next Halpern update of w and A^* y, then Q w of the
    new iterate with the next step's elementwise pass): the bar iterates after 100, 200 and 300
    steps match the oracle's, normwise and element by element."""
    qp = PROBLEMS[name]
    K = 300
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    with pkg.Solver(qp, lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q) as s:
        for k in (100, 200, 300):
            s.solve(tol=1e-30, max_iter=k)
            x, y, z, w, kkt = s.get()
            # the capped solve ends at step k's stopping test, before its restart decision
            assert kkt["iters"] == k and kkt["restarts"] == int(ref.trace["restart"][:k - 1].sum()), (name, k)
            ex = close(x, ref.trace["x"][k - 1])
            assert ex <= ITER_TOL, (name, k, ex)
            if qp.qterms:   # w_Q lives in Range(Q): with Q = 0 the library never forms it
                assert close(w, ref.trace["w"][k - 1]) <= ITER_TOL, (name, k)
            if qp.m:
                ey = close(y, ref.trace["y"][k - 1])
                assert ey <= ITER_TOL, (name, k, ey)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_converged_objective(pkg, name):
    qp = PROBLEMS[name]
    ref = oracle.solve(qp, tol=1e-8, max_iter=500000)
    assert ref.status == "converged"
    with pkg.Solver(qp, lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q) as s:
        st = s.solve(tol=1e-8, max_iter=500000)
        x, y, z, w, kkt = s.get()
    assert st == "converged", kkt
    assert abs(kkt["pobj"] - ref.pobj) <= OBJ_TOL * (1 + abs(ref.pobj))
    # the GPU's own stopping test is honest: recompute eta on its output with the oracle
    e, _, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.05e-8, e
    assert np.all(x >= qp.L) and np.all(x <= qp.U)


def test_power_method(pkg):
    qp = PROBLEMS["plain"]
    from tests import dense_ref as D
    A, Q = D.dense_of(qp)
    la = np.linalg.eigvalsh(A @ A.T).max()
    lq = np.linalg.eigvalsh(Q).max()
    with pkg.Solver(qp) as s:
        s.solve(tol=1e-30, max_iter=1)
        k = s.kkt()
    assert la <= k["lambda_A"] <= 1.01 * la * (1 + 1e-6)
    assert lq <= k["lambda_Q"] <= 1.01 * lq * (1 + 1e-6)
    ref = oracle.solve(qp, max_iter=1)
    assert abs(k["lambda_A"] - ref.lambda_A) <= 1e-5 * ref.lambda_A
    assert abs(k["lambda_Q"] - ref.lambda_Q) <= 1e-5 * ref.lambda_Q


def test_power_methods_side_by_side_match_each_alone(pkg):
    # with A and Q both present the two power methods run at once on two streams, each with its
    # own state; run alone (the other lambda given) each must give the same value bit for bit,
    # and a second solve on the same handle must repeat it (the state is reset per solve)
    qp = PROBLEMS["plain"]
    with pkg.Solver(qp) as s:
        s.solve(tol=1e-30, max_iter=1)
        both = s.kkt()
        s.solve(tol=1e-30, max_iter=1)
        again = s.kkt()
    assert (again["lambda_A"], again["lambda_Q"]) == (both["lambda_A"], both["lambda_Q"])
    with pkg.Solver(qp, lambda_Q=both["lambda_Q"]) as s:
        s.solve(tol=1e-30, max_iter=1)
        assert s.kkt()["lambda_A"] == both["lambda_A"]
    with pkg.Solver(qp, lambda_A=both["lambda_A"]) as s:
        s.solve(tol=1e-30, max_iter=1)
        assert s.kkt()["lambda_Q"] == both["lambda_Q"]


def test_default_run_matches_oracle_objective(pkg):
    # both sides estimate lambda themselves (power method), defaults everywhere
    qp = qpgen.plain_cqp()
    ref = oracle.solve(qp, tol=1e-8, max_iter=200000)
    with pkg.Solver(qp) as s:
        assert s.solve(tol=1e-8, max_iter=200000) == "converged"
        k = s.kkt()
    assert abs(k["pobj"] - ref.pobj) <= OBJ_TOL * (1 + abs(ref.pobj))
    assert k["rel_kkt"] <= 1e-8


def test_warm_start(pkg):
    qp = PROBLEMS["plain"]
    x0 = np.clip(np.random.default_rng(3).random(qp.n), qp.L, qp.U)
    y0 = np.random.default_rng(4).standard_normal(qp.m) * 0.1
    ref = oracle.solve(qp, tol=1e-30, max_iter=40, x0=x0, y0=y0, trace_len=40)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        s.set_warm_start(x0, y0)
        for k in (1, 15, 40):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL
            assert close(y, ref.trace["y"][k - 1]) <= ITER_TOL


def test_halpern_total_and_golden_section(pkg):
    # Options: Halpern weights from the total counter (Algorithm 4 as printed) and the
    # golden-section search of Algorithm 5.  Golden section compares f at two points whose
    # values differ by less than the rounding of f once the bracket is narrow, so sigma
    # agrees only to about 1e-9 between two correct implementations; the bound here is 1e-8.
    qp = PROBLEMS["plain"]
    ref = oracle.solve(qp, tol=1e-30, max_iter=40, trace_len=40, halpern_total=1, sigma_golden=1)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q, halpern_total=1, sigma_golden=1) as s:
        for k in (1, 15, 40):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= 1e-8
            assert close(y, ref.trace["y"][k - 1]) <= 1e-8
    # exact argmin with the total-counter weights keeps the tight bound
    ref = oracle.solve(qp, tol=1e-30, max_iter=40, trace_len=40, halpern_total=1)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q, halpern_total=1) as s:
        for k in (15, 40):
            s.solve(tol=1e-30, max_iter=k)
            x, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL


def test_invalid_arguments(pkg):
    qp = qpgen.random_small(n=5, m=3, seed=1)
    bad = qpgen.QP(**{**qp.__dict__, "l": qp.u + 1})
    with pytest.raises(pkg.HPRQPError) as e:
        pkg.Solver(bad)
    assert e.value.status == 4
    c = qp.c.copy(); c[1] = np.nan
    with pytest.raises(pkg.HPRQPError):
        pkg.Solver(qpgen.QP(**{**qp.__dict__, "c": c}))
    ci = qp.A_colidx.copy(); ci[-1] = 99
    with pytest.raises(pkg.HPRQPError):
        pkg.Solver(qpgen.QP(**{**qp.__dict__, "A_colidx": ci}))
    # an infinite bound on the wrong side (l = u = +inf is an empty row set, Sec. 1); the
    # other bound moves with it, so that lo <= hi still holds
    for lo, hi, idx, v in (("l", "u", 0, np.inf), ("l", "u", 2, -np.inf),
                           ("L", "U", 1, np.inf), ("L", "U", 3, -np.inf)):
        a, b = getattr(qp, lo).copy(), getattr(qp, hi).copy()
        a[idx] = b[idx] = v
        with pytest.raises(pkg.HPRQPError) as e:
            pkg.Solver(qpgen.QP(**{**qp.__dict__, lo: a, hi: b}))
        assert e.value.status == 4, (lo, v)
    with pkg.Solver(qp) as s:
        with pytest.raises(pkg.HPRQPError):
            s.solve(tol=1e-8, max_iter=0)
        with pytest.raises(pkg.HPRQPError):
            s.solve(tol=-1.0, max_iter=10)
        l_bad, u_bad = qp.l.copy(), qp.u.copy()
        l_bad[0] = u_bad[0] = np.inf
        with pytest.raises(pkg.HPRQPError):
            s.set_data(l=l_bad, u=u_bad)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_launch_modes_agree(pkg, mode):
    # the flat graph (variants read inside the kernels) and host-driven stream launches run the
    # same algorithm as the conditional graph: identical iterates up to rounding
    qp = PROBLEMS["large_sum"]
    ref = oracle.solve(qp, tol=1e-30, max_iter=60, trace_len=60)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q, launch_mode=mode) as s:
        for k in (7, 60):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL
            assert close(y, ref.trace["y"][k - 1]) <= ITER_TOL
        st = s.solve(tol=1e-8, max_iter=100000)
        assert st == "converged"


def test_tolerance_ladder(pkg):
    """Iterations and time to 1e-4 and 1e-6 recorded during a 1e-8 solve (Sec. 4 reports the
    three tolerances): they are where looser solves stop, and the oracle's."""
    qp = PROBLEMS["plain"]
    ref = oracle.solve(qp, tol=1e-8, max_iter=500000)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        assert s.solve(tol=1e-8, max_iter=500000) == "converged"
        k = s.kkt()
        assert 0 < k["iters_1e4"] <= k["iters_1e6"] <= k["iters"]
        assert 0 < k["seconds_1e4"] <= k["seconds_1e6"] <= k["solve_seconds"] * 1.01 + 1e-3
        assert (k["iters_1e4"], k["iters_1e6"]) == (ref.iters_1e4, ref.iters_1e6)
        for tol, key in ((1e-4, "iters_1e4"), (1e-6, "iters_1e6")):
            assert s.solve(tol=tol, max_iter=500000) == "converged"
            assert s.kkt()["iters"] == k[key]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_persistent_solver_matches_oracle(pkg, name):
    """launch_mode 3 (every pass of many steps in one cooperative launch, grid barriers between
    passes) reproduces the oracle's iterates and converged objective on every family."""
    qp = PROBLEMS[name]
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    lam = dict(lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q)
    with pkg.Solver(qp, launch_mode=3, **lam) as s:
        for k in (1, 2, 11, 21, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL, k
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= ITER_TOL, k
    full = oracle.solve(qp, tol=1e-8, max_iter=500000)
    with pkg.Solver(qp, launch_mode=3, lambda_A=full.lambda_A if qp.m else 0.0, lambda_Q=full.lambda_Q) as s:
        assert s.solve(tol=1e-8, max_iter=500000) == "converged"
        x, y, z, w, kkt = s.get()
    assert abs(kkt["pobj"] - full.pobj) <= OBJ_TOL * (1 + abs(full.pobj))
    e, _, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.05e-8, e


def test_stopping_test_history(pkg):
    """Every stopping test of a solve is recorded on the device (iteration, restarts, sigma,
    eta's, objectives, R~, device time); the last one is the solve's result."""
    qp = PROBLEMS["plain"]
    with pkg.Solver(qp) as s:
        assert s.solve(tol=1e-8, max_iter=500000) == "converged"
        k = s.kkt()
        hist = s.history()
    assert len(hist) == min(512, k["iters"] // 100)
    assert [h["iter"] for h in hist] == list(range(k["iters"] - 100 * (len(hist) - 1), k["iters"] + 1, 100))
    last = hist[-1]
    for key in ("eta_p", "eta_d", "eta_gap", "pobj", "dobj", "sigma"):
        assert last[key] == k[key], key
    assert last["restarts"] == k["restarts"]
    secs = [h["seconds"] for h in hist]
    assert all(b >= a for a, b in zip(secs, secs[1:])) and secs[0] > 0
    assert max(last["eta_p"], last["eta_d"], last["eta_gap"]) <= 1e-8


def _long_and_empty_rows():
    """n = 1500: Q = diag(d) + u u^T stored as CSR (every row 1500 entries, so each row spans
    two staging windows of 1024 entries), A with one dense row, five empty rows and a ragged
    tail past the last full chunk of 256 rows."""
    rng = np.random.default_rng(11)
    n, m = 1500, 300
    uu = rng.standard_normal(n) / np.sqrt(n)
    Q = np.diag(rng.uniform(0.5, 1.5, n)) + np.outer(uu, uu)
    A = np.where(rng.random((m, n)) < 0.01, rng.standard_normal((m, n)), 0.0)
    A[0] = 1.0
    A[5:10] = 0.0
    return qpgen.from_dense(Q, rng.standard_normal(n), A=A, l=np.full(m, -1.0), u=np.full(m, 1.0),
                            L=np.full(n, -2.0), U=np.full(n, 2.0))


STAGED = dict(PROBLEMS, long_rows=_long_and_empty_rows())


@pytest.mark.parametrize("tune", [2, 3])
@pytest.mark.parametrize("name", list(STAGED))
def test_staged_schedule_matches_oracle(pkg, name, tune):
    """autotune = 2 runs every CSR pass in the staged chunk form (the block streams a chunk's
    entries in windows, then each thread sums its own row); autotune = 3 runs the A and A^T
    passes from their SELL-32 copies (one row per lane, rows sorted by length inside each
    256-row chunk): same products and iterates."""
    qp = STAGED[name]
    rng = np.random.default_rng(1)
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    with pkg.Solver(qp, autotune=tune, lambda_A=ref.lambda_A if qp.m else 0.0, lambda_Q=ref.lambda_Q) as s:
        v = rng.standard_normal(qp.n)
        assert rel(s.apply("Q", v), oracle.qmul(qp, v)) <= 1e-13
        if qp.m:
            yv = rng.standard_normal(qp.m)
            assert rel(s.apply("A", v), oracle.amul(qp, v)) <= 1e-13
            assert rel(s.apply("AT", yv), oracle.atmul(qp, yv)) <= 1e-13
        for k in (1, 11, 21, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= ITER_TOL, (name, k)
            if qp.m:
                assert close(y, ref.trace["y"][k - 1]) <= ITER_TOL, (name, k)


@pytest.mark.parametrize("name", ["plain", "large_sum", "lasso"])
def test_programmatic_launches_change_nothing(pkg, name):
    """The step kernels as programmatic dependent launches (the default) reach bit-identical
    iterates to ordinary launches: each kernel still waits for its predecessor's results.
    (Both handles take the schedule from the row lengths: the timed autotuner may pick
    different lanes per row for two handles, which changes the rounding.)"""
    qp = PROBLEMS[name]
    out = []
    for pdl in (1, 0):
        with pkg.Solver(qp, pdl=pdl, autotune=0) as s:
            s.solve(tol=1e-30, max_iter=333)
            x, y, z, w, k = s.get()
            out.append((x, y, k["iters"], k["restarts"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]


@pytest.mark.parametrize("name,extra", [("plain", {}), ("large_sum", {}), ("lasso", {}), ("csrQ", {}),
                                        ("plain", {"sigma_fixed": 1}), ("plain", {"restart_off": 1}),
                                        ("plain", {"check_every": 30, "restart_every": 7})])
def test_fixed_schedule_graph_matches_dynamic_graph(pkg, name, extra):
    """Whole periods through the fixed-schedule graph (one conditional node per R~ test) and
    the tail through the dynamic graph give bit-identical iterates, restarts and stopping
    values to running every step through the dynamic graph when every step runs its five
    passes (fused_steps = 0).  With the fused passes (the default) Q w is formed directly
    instead of through the Halpern recurrence of its image, so the iterates agree to rounding
    (1e-11 relative, element by element) with the same iterations, restarts and status.  sigma
    agrees to 1e-5 only: Algorithm 5 forms theta~ from differences of nearly equal iterates late
    in a solve, which magnifies the rounding differences of the two paths (a logic error would
    change the iteration or restart counts, which must match exactly)."""
    qp = PROBLEMS[name]
    for tol, it in ((1e-30, 333), (1e-8, 200000)):
        out = []
        for fixed, fused in ((1, 0), (0, 1), (1, 1)):
            with pkg.Solver(qp, fixed_schedule=fixed, fused_steps=fused, autotune=0, **extra) as s:
                st = s.solve(tol=tol, max_iter=it)
                x, y, z, w, k = s.get()
                out.append((st, x, y, k["iters"], k["restarts"], k["sigma"], k["pobj"], k["rel_kkt"]))
        assert out[0][0] == out[1][0]
        assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
        assert out[0][3:] == out[1][3:], (out[0][3:], out[1][3:])
        f = out[2]
        assert f[0] == out[1][0] and f[3:5] == out[1][3:5], (f[3:5], out[1][3:5])
        assert close(f[1], out[1][1]) <= 1e-11 and close(f[2], out[1][2]) <= 1e-11
        assert abs(f[5] - out[1][5]) <= 1e-5 * out[1][5]
        assert abs(f[6] - out[1][6]) <= 1e-9 * (1 + abs(out[1][6]))
