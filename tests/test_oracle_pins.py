"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed-form solutions,
brute-force active-set enumeration, an LP library, the subproblem optimality conditions
written from their definitions, the dense metric M of eq. (2.12), Algorithm 2 with an
explicit range-space basis (Thm. 3.1), the O(1/k) bound of Thm. 3.2, and the printed
parameter values of Sec. 4.1.
"""
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import oracle
import qpgen
from tests import dense_ref as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _solve(qp, **kw):
    kw.setdefault("tol", 1e-10)
    kw.setdefault("max_iter", 400000)
    return oracle.solve(qp, **kw)


# ------------------------------------------------------------------ closed forms
def test_unconstrained_closed_form():
    # m = 0, C = R^n, Q > 0: the minimiser is -Q^{-1} c (Sec. 1, eq. (1.1) with phi = 0)
    rng = np.random.default_rng(1)
    n = 12
    F = rng.standard_normal((n, n))
    Q = F.T @ F + 0.5 * np.eye(n)
    c = rng.standard_normal(n)
    qp = qpgen.from_dense(Q, c)
    s = _solve(qp)
    assert s.status == "converged"
    x = np.linalg.solve(Q, -c)
    assert np.linalg.norm(s.x - x) <= 1e-7 * max(1, np.linalg.norm(x))


def test_diag_box_closed_form():
    # diagonal Q, box only: separable, x_j = clip(-c_j/q_j, L_j, U_j)
    rng = np.random.default_rng(2)
    n = 30
    q = rng.uniform(0.5, 3.0, n)
    c = 3 * rng.standard_normal(n)
    L = -rng.random(n)
    U = rng.random(n)
    qp = qpgen.from_dense(np.diag(q), c, L=L, U=U, q_kind="diag")
    s = _solve(qp)
    assert s.status == "converged"
    np.testing.assert_allclose(s.x, np.clip(-c / q, L, U), atol=1e-8)
    # x bar lies in C exactly (it is a projection, eq. (3.2))
    assert np.all(s.x >= L) and np.all(s.x <= U)


def test_l1_orthonormal_design_soft_threshold():
    # Lasso with orthonormal design (Sec. 4.4): Q = F^T F = I, c = -F^T b, the minimiser of
    # 1/2||x||^2 - <F^T b, x> + lam||x||_1 is soft(F^T b, lam)
    rng = np.random.default_rng(3)
    n = 16
    F, _ = np.linalg.qr(rng.standard_normal((n, n)))
    b = rng.standard_normal(n)
    g = F.T @ b
    lam = 0.4
    qp = qpgen.QP(n, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), -g, np.zeros(0),
                  np.zeros(0), np.full(n, -np.inf), np.full(n, np.inf), qpgen.PHI_L1, lam,
                  [qpgen.QTerm("dense_factor", p=n, dense=np.ascontiguousarray(F))])
    s = _solve(qp)
    assert s.status == "converged"
    np.testing.assert_allclose(s.x, np.sign(g) * np.maximum(np.abs(g) - lam, 0), atol=1e-8)
    # eq. (3.1) with the Moreau identity: zbar lies in [-lam, lam] by construction
    assert np.all(np.abs(s.z) <= lam * (1 + 1e-12))


def test_l1_box_separable():
    # lam|x| + box with diagonal Q: per coordinate clip(soft(-c/q... )) -> compute by 1-D
    # minimisation on a fine grid refined analytically: x = clip(soft(-c, lam)/q, L, U)
    rng = np.random.default_rng(4)
    n = 20
    q = rng.uniform(0.5, 2.0, n)
    c = 2 * rng.standard_normal(n)
    L = -0.5 * rng.random(n) - 0.1
    U = 0.5 * rng.random(n) + 0.1
    lam = 0.3
    qp = qpgen.from_dense(np.diag(q), c, L=L, U=U, phi="l1_box", lam=lam, q_kind="diag")
    s = _solve(qp)
    assert s.status == "converged"
    soft = np.sign(-c) * np.maximum(np.abs(c) - lam, 0)
    np.testing.assert_allclose(s.x, np.clip(soft / q, L, U), atol=1e-8)


def test_l1_with_unbounded_sides_closed_form():
    """lam|x| + the indicator of [L, U] with infinite sides (x >= 0 as in a nonnegative Lasso,
    x <= U, and both sides free), diagonal Q: the solution is clip(soft(-c, lam)/q, L, U)
    coordinate by coordinate, and the solve must stop on the Sec. 4.1 rule (the dual value
    phi*(-zbar) stays finite on the unbounded sides)."""
    rng = np.random.default_rng(7)
    n = 40
    q = rng.uniform(0.5, 2.0, n)
    c = 2 * rng.standard_normal(n)
    L = np.where(np.arange(n) % 4 == 0, 0.0, -np.inf)
    U = np.where(np.arange(n) % 4 == 1, 0.4, np.inf)
    L[2::4], U[2::4] = -0.3, 0.3
    lam = 0.3
    qp = qpgen.from_dense(np.diag(q), c, L=L, U=U, phi="l1_box", lam=lam, q_kind="diag")
    s = _solve(qp)
    assert s.status == "converged"
    soft = np.sign(-c) * np.maximum(np.abs(c) - lam, 0)
    xs = np.clip(soft / q, L, U)
    np.testing.assert_allclose(s.x, xs, atol=1e-8)
    assert np.count_nonzero(xs[L == 0.0] > 0) >= 3     # interior points on a side with U = inf
    p_star = 0.5 * q @ xs**2 + c @ xs + lam * np.abs(xs).sum()
    assert s.pobj == pytest.approx(p_star, rel=1e-8)


def test_l1_box_conjugate_on_unbounded_sides():
    """phi*(-z) for lam|x| + the indicator of [L, U] (the Sec. 4.1 dual objective): per
    coordinate sup over [L, U] of (-z x - lam|x|), finite only for z <= lam where L = -inf and
    z >= -lam where U = +inf.  A z a few ulps past that edge (rounding of zbar) is taken on the
    edge; a z further out gives +inf, i.e. the dual value -inf."""
    lam = 0.5
    L = np.array([-np.inf, 0.0, -1.0])
    U = np.array([1.0, np.inf, 2.0])
    qp = qpgen.from_dense(np.eye(3), np.zeros(3), L=L, U=U, phi="l1_box", lam=lam, q_kind="diag")
    x = np.zeros(3)
    z_edge = np.array([lam, -lam, -0.7])
    # closed form per coordinate: max over the finite end points and 0 (0 lies in every [L, U])
    expect = -(0.0 + 0.0 + max(0.7 * -1.0 - lam * 1.0, 0.7 * 2.0 - lam * 2.0, 0.0))
    _, _, d_edge = oracle.eta(qp, x, np.zeros(0), z_edge)
    assert d_edge == pytest.approx(expect, abs=1e-15)
    z_ulp = np.array([np.nextafter(lam, 1.0), np.nextafter(-lam, -1.0), -0.7])
    _, _, d_ulp = oracle.eta(qp, x, np.zeros(0), z_ulp)
    assert d_ulp == d_edge
    for z_far in (np.array([lam + 1e-6, -lam, -0.7]), np.array([lam, -lam - 1e-6, -0.7])):
        _, _, d_far = oracle.eta(qp, x, np.zeros(0), z_far)
        assert np.isneginf(d_far), d_far


def test_lp_special_case_matches_linprog():
    # Q = 0, phi = delta_C: HPR-QP reduces to HPR-LP (Sec. 2.2 remark); compare the
    # optimal value with an LP library (HiGHS through scipy)
    rng = np.random.default_rng(5)
    n, m = 10, 6
    A = rng.standard_normal((m, n))
    x0 = rng.random(n)
    l = A @ x0 - rng.random(m)
    u = A @ x0 + rng.random(m)
    l[:2] = u[:2] = (A @ x0)[:2]
    c = rng.standard_normal(n)
    qp = qpgen.from_dense(None, c, A=A, l=l, u=u, L=np.zeros(n), U=np.ones(n))
    s = _solve(qp)
    assert s.status == "converged"
    A_ub = np.vstack([A[2:], -A[2:]])
    b_ub = np.concatenate([u[2:], -l[2:]])
    ref = so.linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A[:2], b_eq=l[:2], bounds=list(zip([0] * n, [1] * n)),
                     method="highs")
    assert ref.status == 0
    assert abs(s.pobj - ref.fun) <= 1e-7 * (1 + abs(ref.fun))
    assert s.lambda_Q == 0.0


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed,q_kind,rank", [(0, "csr", None), (1, "csr", None), (2, "factor", 2),
                                              (3, "dense_factor", 3), (4, "factor", 1), (5, "csr", None)])
def test_brute_force_active_sets(seed, q_kind, rank):
    qp = qpgen.random_small(n=5, m=3, seed=seed, q_kind=q_kind, q_rank=rank)
    best = D.brute_force(qp)
    assert best is not None
    obj, xs, ys, zs = best
    s = _solve(qp, tol=1e-10)
    assert s.status == "converged"
    assert abs(s.pobj - obj) <= 1e-8 * (1 + abs(obj))
    if rank is None:  # Q > 0: the minimiser is unique
        np.testing.assert_allclose(s.x, xs, atol=1e-6)
    # the brute-force point is a KKT point: eta vanishes there (Sec. 4.1 definitions)
    e, _, _ = oracle.eta(qp, xs, ys, zs)
    assert np.max(e) <= 1e-10


def test_kkt_invariants_at_termination():
    qp = qpgen.plain_cqp(n=200, m=100, seed=7, q_rows=20, a_density=0.05, q_density=0.1)
    s = _solve(qp, tol=1e-8)
    assert s.status == "converged"
    assert max(s.eta_p, s.eta_d, s.eta_gap) <= 1e-8
    # xbar = Prox (a projection onto C): in C exactly
    assert np.all(s.x >= qp.L) and np.all(s.x <= qp.U)
    # ybar of eq. (3.5): positive only at a finite lower bound, negative at a finite upper
    assert np.all(~((s.y > 0) & ~np.isfinite(qp.l)))
    assert np.all(~((s.y < 0) & ~np.isfinite(qp.u)))
    # zbar of eq. (3.1): zbar_j > 0 only where xbar_j = L_j, < 0 only where xbar_j = U_j
    assert np.all((s.z <= 0) | (s.x == qp.L))
    assert np.all((s.z >= 0) | (s.x == qp.U))
    # eta recomputed independently of the iteration agrees with the reported one
    e, _, _ = oracle.eta(qp, s.x, s.y, s.z)
    np.testing.assert_allclose(e, [s.eta_p, s.eta_d, s.eta_gap], rtol=1e-12, atol=1e-300)


# ------------------------------------------------------------------ metric M, eq. (2.12)
@pytest.mark.parametrize("rank", [None, 2])
def test_mnorm_matches_dense_metric(rank):
    qp = qpgen.random_small(n=6, m=4, seed=11, q_kind="csr" if rank is None else "factor", q_rank=rank)
    A, Q = D.dense_of(qp)
    lamA = 1.01 * np.linalg.eigvalsh(A @ A.T).max()
    lamQ = 1.01 * np.linalg.eigvalsh(Q).max()
    M = D.metric_M(A, Q, 0.7, lamA, lamQ)
    # M is positive semidefinite on R^m x W x R^n x R^n (Assumption 2.2 / Prop. 2.3)
    d, V = D.range_basis(Q)
    m, n = qp.m, qp.n
    P = np.zeros((m + 3 * n, m + d.size + 2 * n))
    P[:m, :m] = np.eye(m)
    P[m:m + n, m:m + d.size] = V
    P[m + n:, m + d.size:] = np.eye(2 * n)
    assert np.linalg.eigvalsh(P.T @ M @ P).min() >= -1e-9 * np.abs(M).max()
    rng = np.random.default_rng(0)
    for sigma in (0.05, 0.7, 9.0):
        for _ in range(3):
            dy, dw, dx = rng.standard_normal(m), rng.standard_normal(n), rng.standard_normal(n)
            ref = D.mnorm2_dense(A, Q, sigma, lamA, lamQ, dy, dw, dx)
            got = oracle.mnorm2(qp, sigma, lamA, lamQ, dy, dw, dx)
            assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref))


# ------------------------------------------------------------------ one step: subproblem optimality
def _support_subgrad_ok(s, y, lo, hi, tol):
    """s in d delta*_K(-y): s in [lo, hi], s = lo where y > 0, s = hi where y < 0."""
    ok = np.all(s >= lo - tol) & np.all(s <= hi + tol)
    ok &= np.all(np.where(y > tol, np.abs(s - lo) <= tol, True))
    ok &= np.all(np.where(y < -tol, np.abs(s - hi) <= tol, True))
    return bool(ok)


@pytest.mark.parametrize("seed,rank", [(21, None), (22, 2), (23, 3)])
def test_one_step_subproblem_optimality(seed, rank):
    """Steps 1-3 of Algorithm 3 solve the subproblems of Algorithm 2 (Prop. 3.1, eq. (2.11)):
    each optimality condition, written from L_sigma and the proximal terms, holds."""
    qp = qpgen.random_small(n=6, m=4, seed=seed, q_kind="csr" if rank is None else "factor", q_rank=rank)
    A, Q = D.dense_of(qp)
    rng = np.random.default_rng(seed)
    lamA = 1.01 * np.linalg.eigvalsh(A @ A.T).max()
    lamQ = 1.01 * np.linalg.eigvalsh(Q).max()
    sigma = 0.8
    y, w, x = rng.standard_normal(qp.m), rng.standard_normal(qp.n), rng.standard_normal(qp.n)
    yb, wb, zb, xb, wh = oracle.step(qp, sigma, lamA, lamQ, y, w, x)
    c = qp.c
    tol = 1e-10
    # Step 1: 0 in -d phi*(-zb) + x + sigma(-Qw + A^*y + zb - c); the point in the
    # subdifferential is xbar (Step 2), so xbar must satisfy Step 2 exactly and -zb in
    # d delta_C(xbar): xbar in C, zb > 0 only at L, zb < 0 only at U
    np.testing.assert_allclose(xb, x + sigma * (-Q @ w + A.T @ y + zb - c), atol=1e-12)
    assert np.all(xb >= qp.L) and np.all(xb <= qp.U)
    assert np.all((zb <= tol) | (np.abs(xb - qp.L) <= tol))
    assert np.all((zb >= -tol) | (np.abs(xb - qp.U) <= tol))
    # Step 3-1 on W (gradient of the w-subproblem, all terms in Range(Q)):
    # Q[wh - xb + sigma(Q wh - A^*y - zb + c)] + sigma Q(lamQ I - Q)(wh - w) = 0
    g1 = Q @ (wh - xb + sigma * (Q @ wh - A.T @ y - zb + c)) + sigma * Q @ (lamQ * wh - Q @ wh - lamQ * w + Q @ w)
    assert np.linalg.norm(g1) <= 1e-10
    # Step 3-2: 0 in -d delta*_K(-yb) + A xb + sigma A(-Q wh + A^* yb + zb - c) + sigma S_y (yb - y)
    s = A @ xb + sigma * A @ (-Q @ wh + A.T @ yb + zb - c) + sigma * (lamA * (yb - y) - A @ A.T @ (yb - y))
    assert _support_subgrad_ok(s, yb, qp.l, qp.u, 1e-9)
    # Step 3-3: like 3-1 with yb
    g3 = Q @ (wb - xb + sigma * (Q @ wb - A.T @ yb - zb + c)) + sigma * Q @ (lamQ * wb - Q @ wb - lamQ * w + Q @ w)
    assert np.linalg.norm(g3) <= 1e-10


@pytest.mark.parametrize("seed,rank", [(31, None), (32, 2)])
def test_sgs_joint_step(seed, rank):
    """Prop. 2.3: the sGS sequence w1/2 -> y -> w solves the joint (y, w) step of
    Algorithm 1 with T1 = S + S_sGS (eqs. (2.6)-(2.7), S_sGS from its definition)."""
    qp = qpgen.random_small(n=6, m=4, seed=seed, q_kind="csr" if rank is None else "factor", q_rank=rank)
    A, Q = D.dense_of(qp)
    rng = np.random.default_rng(seed)
    lamA = 1.01 * np.linalg.eigvalsh(A @ A.T).max()
    lamQ = 1.01 * np.linalg.eigvalsh(Q).max()
    sigma = 1.3
    y, w, x = rng.standard_normal(qp.m), rng.standard_normal(qp.n), rng.standard_normal(qp.n)
    d, V = D.range_basis(Q)
    w = V @ (V.T @ w)  # w^k in W
    yb, wb, zb, xb, wh = oracle.step(qp, sigma, lamA, lamQ, y, w, x)
    wbW = V @ (V.T @ wb)  # Pi_W(wb): same Q-image (Prop. 3.1)
    np.testing.assert_allclose(Q @ wbW, Q @ wb, atol=1e-10)
    M = D.metric_M(A, Q, sigma, lamA, lamQ)
    m, n = qp.m, qp.n
    # T1 = M[yw,yw] - sigma A_Q^* A_Q
    AQ = np.hstack([A.T, -Q])
    T1 = M[:m + n, :m + n] - sigma * AQ.T @ AQ
    dyw = np.concatenate([yb - y, wbW - w])
    T1d = T1 @ dyw
    c = qp.c
    # y-block: 0 in -d delta*_K(-yb) + A xb + sigma A(-Q wb + A^* yb + zb - c) + (T1 d)_y
    s = A @ xb + sigma * A @ (-Q @ wbW + A.T @ yb + zb - c) + T1d[:m]
    assert _support_subgrad_ok(s, yb, qp.l, qp.u, 1e-9)
    # w-block, projected on W: Q wb - Q xb - sigma Q(-Q wb + A^*yb + zb - c) + (T1 d)_w
    gw = Q @ wbW - Q @ xb - sigma * Q @ (-Q @ wbW + A.T @ yb + zb - c) + T1d[m:]
    assert np.linalg.norm(V.T @ gw) <= 1e-9


# ------------------------------------------------------------------ Thm. 3.1
@pytest.mark.parametrize("seed,rank", [(41, 2), (42, 3), (43, None)])
def test_thm31_shadow_sequence_equals_alg2(seed, rank):
    """Algorithm 3 (shadow w_Q, no projection) and Algorithm 2 (every w-step a minimisation
    over W = Range(Q)) produce the same (ybar, Q wbar, zbar, xbar) from the origin."""
    qp = qpgen.random_small(n=6, m=4, seed=seed, q_kind="csr" if rank is None else "factor", q_rank=rank)
    A, Q = D.dense_of(qp)
    lamA = 1.01 * np.linalg.eigvalsh(A @ A.T).max()
    lamQ = 1.01 * np.linalg.eigvalsh(Q).max()
    sigma = 0.6
    K = 25
    ref = D.alg2_run(qp, sigma, lamA, lamQ, K)
    n, m = qp.n, qp.m
    y, w, x = np.zeros(m), np.zeros(n), np.zeros(n)
    for k in range(K):
        yb, wb, zb, xb, _ = oracle.step(qp, sigma, lamA, lamQ, y, w, x)
        ry, rQw, rz, rx = ref[k]
        scale = 1 + np.abs(np.concatenate([ry, rQw, rz, rx])).max()
        assert np.abs(yb - ry).max() <= 1e-9 * scale
        assert np.abs(Q @ wb - rQw).max() <= 1e-9 * scale
        assert np.abs(zb - rz).max() <= 1e-9 * scale
        assert np.abs(xb - rx).max() <= 1e-9 * scale
        a, b = 1.0 / (k + 2), (k + 1.0) / (k + 2)
        y, w, x = b * (2 * yb - y), b * (2 * wb - w), b * (2 * xb - x)
    # the oracle's own loop (fixed sigma, no restart) reproduces the same xbar trajectory
    s = oracle.solve(qp, tol=1e-30, max_iter=K, lambda_A=lamA, lambda_Q=lamQ, sigma0=sigma,
                     restart_off=1, sigma_fixed=1, trace_len=K, scaling=0)
    for k in range(K):
        np.testing.assert_allclose(s.trace["x"][k], ref[k][3], atol=1e-9 * (1 + np.abs(ref[k][3]).max()))


# ------------------------------------------------------------------ Thm. 3.2 (O(1/k))
@pytest.mark.parametrize("seed", [51, 52])
def test_complexity_bound(seed):
    """||ubar^{k+1} - u^k||_M <= ||u^0 - u*||_M / (k+1) for fixed sigma, no restarts,
    with u* a KKT point found by brute force (Thm. 3.2, first bound)."""
    qp = qpgen.random_small(n=5, m=3, seed=seed, q_kind="factor", q_rank=3)
    A, Q = D.dense_of(qp)
    obj, xs, ys, zs = D.brute_force(qp)
    lamA = 1.01 * np.linalg.eigvalsh(A @ A.T).max()
    lamQ = 1.01 * np.linalg.eigvalsh(Q).max()
    sigma = 0.9
    R0 = np.sqrt(D.mnorm2_dense(A, Q, sigma, lamA, lamQ, -ys, -xs, -xs))  # u0 = 0, w* = x*
    K = 300
    s = oracle.solve(qp, tol=1e-30, max_iter=K, lambda_A=lamA, lambda_Q=lamQ, sigma0=sigma,
                     restart_off=1, sigma_fixed=1, restart_every=1, trace_len=K)
    R = s.trace["R"]
    assert R.size == K and np.all(np.isfinite(R))
    k = np.arange(K)
    assert np.all(R <= R0 / (k + 1) * (1 + 1e-9) + 1e-12)


# ------------------------------------------------------------------ sigma update (Alg. 5)
@pytest.mark.parametrize("t1,t2,t3,lq", [(1.0, 1.0, 0.5, 2.0), (3e-3, 7.0, 40.0, 0.1), (1e-12, 1e-12, 1e-9, 5.0),
                                          (2.0, 0.5, 0.0, 1.0), (1e4, 1e-6, 1e3, 1e3)])
def test_sigma_argmin(t1, t2, t3, lq):
    f = lambda s: t1 * s + t2 / s + s * s * t3 / (1 + lq * s)
    s_exact = oracle.sigma_argmin(t1, t2, t3, lq, golden=False)
    s_gold = oracle.sigma_argmin(t1, t2, t3, lq, golden=True)
    # independent minimiser: bounded Brent on log sigma
    r = so.minimize_scalar(lambda u: f(np.exp(u)), bounds=(np.log(s_exact) - 5, np.log(s_exact) + 5),
                           method="bounded", options={"xatol": 1e-12})
    assert abs(np.log(s_exact) - r.x) <= 1e-5
    assert abs(np.log(s_gold) - np.log(s_exact)) <= 1e-6
    # first-order condition f'(s) = 0 (f strictly convex, eq. (3.10))
    h = 1e-6 * s_exact
    d = (f(s_exact + h) - f(s_exact - h)) / (2 * h)
    assert abs(d) <= 1e-5 * (t1 + t2 / s_exact ** 2 + t3 / lq)
    assert f(s_exact) <= min(f(s_exact * 1.001), f(s_exact / 1.001))


def test_sigma_closed_form_without_theta3():
    # theta3 = 0 (the LP case, Q = 0): f = t1 s + t2/s, argmin sqrt(t2/t1)
    assert oracle.sigma_argmin(4.0, 9.0, 0.0, 0.0) == pytest.approx(1.5, rel=1e-15)


def test_sigma_update_smoothing():
    """Algorithm 5: floors at 1e-12, beta = exp(-R~_{r,tau_r-1}/R~_{0,tau_0-1}) and
    sigma_{r+1} = exp(beta log sigma_new + (1 - beta) log sigma_r)."""
    e = np.e
    # theta3 = 0 and theta1 = theta2: sigma_new = 1, so log sigma_{r+1} = (1 - beta) log sigma_r
    for ratio in (0.0, 0.05, 1.0, 3.0):
        beta = np.exp(-ratio)
        got = oracle.sigma_update(2.0, 2.0, 0.0, 1.0, ratio, e ** 2, False)
        assert np.log(got) == pytest.approx((1 - beta) * 2.0, rel=1e-13, abs=1e-15)
    # ratio 0 (first loop converged to the noise floor): beta = 1, sigma_{r+1} = sigma_new
    assert oracle.sigma_update(4.0, 1.0, 0.0, 1.0, 0.0, 123.0, False) == pytest.approx(0.5, rel=1e-14)
    # floors: tiny theta1, theta2 both become 1e-12, so sigma_new = 1
    assert oracle.sigma_update(1e-30, 1e-40, 0.0, 1.0, 0.0, 7.0, False) == pytest.approx(1.0, rel=1e-14)
    # only theta1, theta2 are floored: theta2 = 4e-12 with theta1 floored gives sqrt(4) = 2
    assert oracle.sigma_update(0.0, 4e-12, 0.0, 1.0, 0.0, 7.0, False) == pytest.approx(2.0, rel=1e-12)


def _sigma_by_derivative_root(t1, t2, t3, lq):
    """argmin of f(s) = t1 s + t2/s + s^2 t3/(1 + lq s) (eq. (3.12)) as the root of
    f'(s) = t1 - t2/s^2 + t3 s (2 + lq s)/(1 + lq s)^2, which increases on s > 0 (f is
    strictly convex, Sec. 3.3), found by scipy's brentq: independent of the oracle's search."""
    fp = lambda s: t1 - t2 / s ** 2 + t3 * s * (2.0 + lq * s) / (1.0 + lq * s) ** 2
    hi = np.sqrt(t2 / t1)          # f'(hi) >= 0: the t3 term is non-negative
    if fp(hi) == 0.0:
        return hi
    lo = hi
    while fp(lo) > 0.0:
        lo *= 0.5
    return so.brentq(fp, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=1000)


@pytest.mark.parametrize("seed,q_kind,rank", [(0, "csr", 3), (1, "factor", 2), (2, "csr", 5), (3, "dense_factor", 1)])
def test_theta_tilde_and_sigma_update_at_every_restart(seed, q_kind, rank):
    """Algorithm 5 at every restart, recomputed from the traced iterates: theta~ of eq. (3.11)
    from the bar iterate ubar^{r,tau_r} of the restarting step and the anchor u^{r,0} (the origin
    for r = 0, then the bar iterate of the previous restart, u^{r+1,0} = ubar^{r,tau_r}), with A and
    Q dense; the floors on theta~_1, theta~_2; the minimiser of eq. (3.12); beta =
    exp(-R~_{r,tau_r-1}/R~_{0,tau_0-1}) and the log-linear smoothing with sigma_r.  A wrong
    anchor (current instead of u^{r,0}) or a sign error in any theta~ term changes sigma_{r+1}."""
    qp = qpgen.random_small(n=7, m=4, seed=seed, q_kind=q_kind, q_rank=rank, eq_rows=1, box=(-1.0, 1.0))
    A, Q = D.dense_of(qp)
    assert np.linalg.matrix_rank(Q) == rank < qp.n   # rank-deficient Q: w lives in Range(Q)
    K = 800
    s = oracle.solve(qp, tol=1e-30, max_iter=K, restart_every=1, check_every=K, trace_len=K, scaling=0)
    tr = s.trace
    lamA, lamQ = s.lambda_A, s.lambda_Q
    rest = [k for k in np.nonzero(tr["restart"])[0] if k + 1 < len(tr["sigma"])]
    assert len(rest) >= 4
    x0, w0, y0 = np.zeros(qp.n), np.zeros(qp.n), np.zeros(qp.m)
    R_first = None
    cross_seen = False
    for k in rest:
        xb, wb, yb = tr["x"][k], tr["w"][k], tr["y"][k]
        dy, dw, dx = yb - y0, wb - w0, xb - x0
        Atdy = A.T @ dy
        th1 = lamA * (dy @ dy) + lamQ * (dw @ Q @ dw) - 2.0 * ((Q @ dw) @ Atdy)
        th2 = dx @ dx
        th3 = Atdy @ Q @ Atdy
        cross_seen |= abs((Q @ dw) @ Atdy) > 1e-6 * max(th1, 1e-12)
        th1, th2 = max(th1, 1e-12), max(th2, 1e-12)
        s_new = _sigma_by_derivative_root(th1, th2, th3, lamQ)
        R = tr["R"][k]
        if R_first is None:
            R_first = R
        beta = np.exp(-(R / R_first if R_first > 0 else 0.0))
        expect = np.exp(beta * np.log(s_new) + (1.0 - beta) * np.log(tr["sigma"][k]))
        assert tr["sigma"][k + 1] == pytest.approx(expect, rel=1e-12), k
        x0, w0, y0 = xb, wb, yb
    assert cross_seen   # the cross term <Q dw, A^* dy> took part in at least one update


# ------------------------------------------------------------------ power method (Sec. 4.1)
def test_power_method_estimates():
    qp = qpgen.plain_cqp(n=300, m=150, seed=3, q_rows=30, a_density=0.05, q_density=0.1)
    A, Q = D.dense_of(qp)
    la = np.linalg.eigvalsh(A @ A.T).max()
    lq = np.linalg.eigvalsh(Q).max()
    ea = oracle.power_A(qp, 5000, 1e-12, 1.0)
    eq = oracle.power_Q(qp, 5000, 1e-12, 1.0)
    assert ea <= la * (1 + 1e-9) and ea >= la * (1 - 1e-6)
    assert eq <= lq * (1 + 1e-9) and eq >= lq * (1 - 1e-6)
    s = oracle.solve(qp, max_iter=1)
    assert s.lambda_A >= la and s.lambda_Q >= lq  # default safety factor keeps lambda >= lambda_1
    # the safety factor: lambda = 1.01 x the estimate, which stops within 1e-4 below lambda_1 here
    assert 1.0099 <= s.lambda_A / la <= 1.0100 + 1e-12
    assert 1.0099 <= s.lambda_Q / lq <= 1.0100 + 1e-12


# ------------------------------------------------------------------ restart bookkeeping (Sec. 3.2)
def test_restart_rules_on_trace():
    qp = qpgen.plain_cqp(n=300, m=150, seed=5, q_rows=30, a_density=0.05, q_density=0.1)
    K = 3000
    s = oracle.solve(qp, tol=1e-30, max_iter=K, restart_every=1, trace_len=K)
    R, rs = s.trace["R"], s.trace["restart"]
    a1, a2 = 0.2, 0.8
    a3 = 0.5
    t = 0
    R0 = Rprev = None
    Rfirst = None
    nrest = 0
    for k in range(K - 1):
        kd = k + 1
        if t == 0:
            expect = False
            R0 = R[k]
        else:
            expect = (R[k] <= a1 * R0) or (R[k] <= a2 * R0 and R[k] > Rprev) or (t + 1 >= a3 * kd)
        Rprev = R[k]
        assert bool(rs[k]) == expect, k
        if expect:
            if Rfirst is None:
                Rfirst = R[k]
            if R[k] / Rfirst <= 0.1:
                a3 = 0.2
            t = 0
            nrest += 1
        else:
            t += 1
    assert nrest >= 5


def test_restart_period_schedule():
    # with restart tests every 10 iterations, restarts happen only at multiples of 10
    qp = qpgen.plain_cqp(n=300, m=150, seed=6, q_rows=30, a_density=0.05, q_density=0.1)
    s = oracle.solve(qp, tol=1e-30, max_iter=2000, restart_every=10, trace_len=2000)
    idx = np.nonzero(s.trace["restart"])[0] + 1
    assert idx.size > 3 and np.all(idx % 10 == 0)
    # R~ is evaluated at multiples of 10 and at the first step of every outer loop
    Rk = np.nonzero(np.isfinite(s.trace["R"]))[0] + 1
    starts = set([1] + list(idx + 1))
    assert set(Rk.tolist()) == set(k for k in range(1, 2001) if k % 10 == 0 or k in starts)


# ------------------------------------------------------------------ printed parameters (Sec. 4.1)
def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_defaults_match_paper():
    g = _golden("paper_parameters.txt")
    p = oracle.default_params()
    for k in ("alpha1", "alpha2", "alpha3", "alpha3_tight", "ratio_tight", "tol"):
        assert p[k] == g[k], k
    assert p["check_every"] == g["check_every"]


def test_sigma0_rule():
    # sigma0 = ||b|| / ||c||, b = max(|l|, |u|) with infinite entries as 0 (Sec. 4.1)
    qp = qpgen.plain_cqp(n=100, m=40, seed=9, q_rows=10, a_density=0.1, q_density=0.1)
    s = oracle.solve(qp, max_iter=1, sigma_fixed=1)
    b = np.maximum(np.where(np.isfinite(qp.l), np.abs(qp.l), 0), np.where(np.isfinite(qp.u), np.abs(qp.u), 0))
    assert s.sigma == pytest.approx(np.linalg.norm(b) / np.linalg.norm(qp.c), rel=1e-14)
    # no rows (b empty, ||b|| = 0 < 1e-16): sigma0 = 1
    las = qpgen.lasso(p=50, q=200, density=0.05)
    assert oracle.solve(las, max_iter=1, sigma_fixed=1).sigma == 1.0


def test_hand_computed_iterates():
    """Three iterations of Algorithm 4 on a 1-D problem computed by hand (golden file)."""
    g = _golden("hand_1d_iterates.txt")
    qp = qpgen.from_dense(np.array([[g["q"]]]), np.array([g["c"]]), L=np.array([g["L"]]), U=np.array([g["U"]]),
                          q_kind="diag")
    for k in range(3):
        s = oracle.solve(qp, tol=1e-30, max_iter=k + 1, lambda_Q=g["lambda_Q"], sigma0=g["sigma"],
                         restart_off=1, sigma_fixed=1, scaling=0)
        assert s.x[0] == pytest.approx(g[f"xbar{k}"], abs=1e-15)
        assert s.z[0] == pytest.approx(g[f"zbar{k}"], abs=1e-15)
        assert s.w[0] == pytest.approx(g[f"wbar{k}"], abs=1e-15)


# ------------------------------------------------------------------ invalid inputs
def test_invalid_inputs_rejected():
    qp = qpgen.random_small(n=4, m=2, seed=1)
    bad = qpgen.QP(**{**qp.__dict__, "l": qp.u + 1.0})
    assert oracle.solve(bad).status == "invalid_arg"
    bad = qpgen.QP(**{**qp.__dict__, "L": qp.U + 1.0})
    assert oracle.solve(bad).status == "invalid_arg"
    c = qp.c.copy(); c[0] = np.nan
    assert oracle.solve(qpgen.QP(**{**qp.__dict__, "c": c})).status == "invalid_arg"
    ci = qp.A_colidx.copy(); ci[0] = qp.n
    assert oracle.solve(qpgen.QP(**{**qp.__dict__, "A_colidx": ci})).status == "invalid_arg"
    assert oracle.solve(qp, max_iter=0).status == "invalid_arg"
    # infinite bounds on the wrong side: l, L in R u {-inf}, u, U in R u {+inf} (Sec. 1);
    # the other bound moves with it, so that lo <= hi still holds
    for lo, hi, idx, v in (("l", "u", 0, np.inf), ("l", "u", 1, -np.inf),
                           ("L", "U", 2, np.inf), ("L", "U", 3, -np.inf)):
        a, b = getattr(qp, lo).copy(), getattr(qp, hi).copy()
        a[idx] = b[idx] = v
        assert oracle.solve(qpgen.QP(**{**qp.__dict__, lo: a, hi: b})).status == "invalid_arg", (lo, v)


def test_tolerance_ladder_marks_where_looser_solves_stop():
    """The ladder iterations are the stopping points of solves run to 1e-4 and 1e-6 (Sec. 4
    reports all three tolerances): the first stopping test that meets each threshold."""
    qp = qpgen.plain_cqp(n=300, m=150, seed=1, q_rows=30, a_density=0.05, q_density=0.1)
    full = oracle.solve(qp, tol=1e-8)
    assert 0 < full.iters_1e4 <= full.iters_1e6 <= full.iters
    assert full.iters_1e4 % 100 == 0 and full.iters_1e6 % 100 == 0
    for tol, k in ((1e-4, full.iters_1e4), (1e-6, full.iters_1e6)):
        s = oracle.solve(qp, tol=tol, lambda_A=full.lambda_A, lambda_Q=full.lambda_Q)
        assert s.status == "converged" and s.iters == k


# ------------------------------------------------------------------ preconditioning (Sec. 4.1)
def _scaled_K(qp, d, e):
    A, Q = D.dense_of(qp)
    n, m = qp.n, qp.m
    K = np.zeros((n + m, n + m))
    K[:n, :n] = Q
    K[n:, :n] = A
    K[:n, n:] = A.T
    s = np.concatenate([d, e])
    return s[:, None] * K * s[None, :], K


@pytest.mark.parametrize("seed,kind", [(61, "csr"), (62, "csr"), (63, "csr")])
def test_pock_chambolle_pass_bounds_the_scaled_norm(seed, kind):
    """After the Pock-Chambolle pass (alpha = 1) the scaled K = [Q A^T; A 0] has spectral
    norm <= 1 (Pock and Chambolle's diagonal preconditioning lemma)."""
    qp = qpgen.random_small(n=7, m=4, seed=seed, q_kind=kind)
    d, e, ok = oracle.scaling(qp)
    assert ok and np.all(d > 0) and np.all(e > 0)
    Ks, K = _scaled_K(qp, d, e)
    assert np.linalg.norm(Ks, 2) <= 1.0 + 1e-12
    # the scaling is not the identity on these badly scaled matrices
    assert not np.allclose(d, 1.0)


def test_scaling_skipped_when_q_is_matrix_free_or_l1():
    assert not oracle.scaling(qpgen.random_small(n=6, m=3, seed=64, q_kind="factor", q_rank=3))[2]
    assert not oracle.scaling(qpgen.qap_relaxation(d=4, seed=1))[2]
    assert not oracle.scaling(qpgen.random_small(n=6, m=3, seed=65, q_kind="csr", phi="l1", lam=0.3))[2]


@pytest.mark.parametrize("seed", [66, 68, 69])
def test_scaled_solve_returns_the_unscaled_solution(seed):
    """Solving the preconditioned problem and mapping back (x = D xs, y = E ys, z = zs / D)
    gives a point that meets the stopping rule of the original problem and has its
    optimal objective (the unscaled solve as reference)."""
    qp = qpgen.random_small(n=8, m=5, seed=seed, q_kind="csr", box=(-1.0, 1.0))
    # stretch the problem's scales so that the preconditioning matters
    rng = np.random.default_rng(seed)
    col = 10.0 ** rng.uniform(-2, 2, qp.n)
    qp.A_vals = qp.A_vals * col[qp.A_colidx]
    a = oracle.solve(qp, tol=1e-10, scaling=1, max_iter=200000)
    b = oracle.solve(qp, tol=1e-10, scaling=0, max_iter=200000)
    assert a.status == b.status == "converged"
    assert a.pobj == pytest.approx(b.pobj, rel=1e-8, abs=1e-9)
    e3, _, _ = oracle.eta(qp, a.x, a.y, a.z)
    assert np.max(e3) <= 1.01e-10
    assert np.all(a.x >= qp.L - 1e-12) and np.all(a.x <= qp.U + 1e-12)
    assert a.iters < b.iters          # on these stretched columns the preconditioning pays


# ------------------------------------------------------------------ primal HPR (Appendix A)
def _primal_1d():
    g = _golden("hand_1d_primal_iterates.txt")
    qp = qpgen.from_dense(np.array([[g["q"]]]), np.array([g["c"]]), A=np.array([[1.0]]),
                          l=np.array([-np.inf]), u=np.array([g["U_row"]]), L=np.array([g["L"]]),
                          U=np.array([g["U"]]))
    return g, qp


@pytest.mark.parametrize("method", [1, 2])
def test_primal_hpr_hand_computed_iterates(method):
    """Algorithms 6 and 7 as printed (fixed sigma, Halpern step, no restart): three iterations
    computed by hand (golden file)."""
    g, qp = _primal_1d()
    for k in range(3):
        s = oracle.solve(qp, tol=1e-30, max_iter=k + 1, method=method, sigma0=g["sigma"],
                         lambda_A=g["lambda_A"], lambda_Q=g["lambda_Q"], scaling=0)
        assert s.x[0] == pytest.approx(g[f"p{method}_xbar{k}"], abs=1e-15)
        assert s.y[0] == pytest.approx(g[f"p{method}_ybar{k}"], abs=1e-15)


@pytest.mark.parametrize("method", [1])
def test_primal_hpr_fixed_point_is_the_kkt_point(method):
    """Started at a KKT point (from a tight HPR-QP solve), Algorithm 6 stays there: the first
    iterate meets the stopping rule (its slack s is not read by Steps 1-3, so (x*, y*) fixes
    the state; Algorithm 7 would also need t = -Q x*, which a warm start does not set)."""
    qp = qpgen.random_small(n=8, m=5, seed=81, q_kind="csr")
    d = oracle.solve(qp, tol=1e-13, max_iter=400000, scaling=0)
    assert d.status == "converged"
    s = oracle.solve(qp, tol=1e-30, max_iter=1, method=method, x0=d.x, y0=d.y, check_every=1, scaling=0)
    assert max(s.eta_p, s.eta_d, s.eta_gap) <= 1e-9
    assert np.allclose(s.x, d.x, atol=1e-9)


def test_primal_hpr_converges_slower_than_hpr_qp():
    """Ablation of Sec. 1's design choices: without restarts and sigma updates the primal
    methods need far more iterations than Algorithm 4 for the same accuracy."""
    qp = qpgen.random_small(n=10, m=6, seed=82, q_kind="csr")
    d = oracle.solve(qp, tol=1e-6, max_iter=400000, scaling=0)
    for method in (1, 2):
        s = oracle.solve(qp, tol=1e-6, max_iter=400000, method=method, scaling=0)
        assert s.status in ("converged", "max_iter")
        assert s.iters > d.iters
        if s.status == "converged":
            assert s.pobj == pytest.approx(d.pobj, rel=1e-4, abs=1e-6)


# ------------------------------------------------------------------ QAP relaxation (Sec. 4.5)
def test_qap_operator_is_the_kronecker_form_and_psd():
    """Q vec(X) = vec(Ahat X Bhat - S X - X T) equals (Bhat (x) Ahat - I (x) S - T (x) I) vec(X)
    (column-major vec), and the LP-derived S, T leave it positive semidefinite."""
    qp = qpgen.qap_relaxation(d=7, seed=3)
    A, Q = D.dense_of(qp)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(qp.n)
        assert np.allclose(oracle.qmul(qp, v), Q @ v, rtol=1e-12, atol=1e-10)
    assert np.linalg.eigvalsh(Q).min() >= -1e-9 * np.abs(Q).max()


def test_qap_bound_lp_value_and_permutation_identity():
    """The (s, t) LP's value is sum_i alpha_i beta_i (alpha descending, beta ascending: the
    rearrangement inequality makes the identity assignment optimal in its dual), and for every
    permutation matrix P the relaxation's objective plus sum(s) + sum(t) is the QAP objective
    tr(Ahat P Bhat P^T)."""
    d = 6
    qp = qpgen.qap_relaxation(d=d, seed=4)
    Ah, Bh = qp.qap_Ahat, qp.qap_Bhat
    alpha = np.sort(np.linalg.eigvalsh(Ah))[::-1]
    beta = np.sort(np.linalg.eigvalsh(Bh))
    assert qp.qap_bound_const == pytest.approx(float(alpha @ beta), rel=1e-9, abs=1e-9)
    _, Q = D.dense_of(qp)
    rng = np.random.default_rng(1)
    for _ in range(5):
        perm = rng.permutation(d)
        P = np.eye(d)[perm]
        x = P.reshape(-1, order="F")
        rel_obj = 0.5 * x @ (Q @ x)               # the solver's objective is 1/2 <x, Qx>, Q = 2 Qhat
        assert rel_obj + qp.qap_bound_const == pytest.approx(np.trace(Ah @ P @ Bh @ P.T), rel=1e-9, abs=1e-9)


def test_qap_relaxation_bound_below_brute_force_optimum():
    """The oracle's optimum of the relaxation plus the LP constant is a lower bound of the QAP
    optimum found by enumerating all permutations (d = 6)."""
    import itertools
    d = 6
    qp = qpgen.qap_relaxation(d=d, seed=5)
    s = oracle.solve(qp, tol=1e-9, max_iter=400000)
    assert s.status == "converged"
    Ah, Bh = qp.qap_Ahat, qp.qap_Bhat
    best = min(np.trace(Ah @ np.eye(d)[list(p)] @ Bh @ np.eye(d)[list(p)].T) for p in itertools.permutations(range(d)))
    qpb = s.pobj + qp.qap_bound_const
    assert qpb <= best + 1e-6
    assert qpb >= qp.qap_bound_const - 1e-6        # Qhat is PSD
    X = s.x.reshape(d, d, order="F")
    assert np.allclose(X.sum(axis=0), 1, atol=1e-6) and np.allclose(X.sum(axis=1), 1, atol=1e-6)


# ------------------------------------------------------------------ operator products
def _dense_by_entries(qp):
    """A and Q assembled entry by entry from the stored arrays, one loop per storage form:
    CSR row i lists (colidx[k], vals[k]) for k in [rowptr[i], rowptr[i+1]); a band term holds
    Q[i][i+o] = Q[i+o][i] = diags[k][i] for offset o = offsets[k]; a factor term (sparse B or
    dense F, p x n) contributes sum over rows r of B[r]^T B[r]; a diagonal term d[j] at (j, j)."""
    n, m = qp.n, qp.m
    A = np.zeros((m, n))
    for i in range(m):
        for k in range(qp.A_rowptr[i], qp.A_rowptr[i + 1]):
            A[i, qp.A_colidx[k]] += qp.A_vals[k]
    Q = np.zeros((n, n))
    for t in qp.qterms:
        if t.kind == "diag":
            for j in range(n):
                Q[j, j] += t.dense[j]
        elif t.kind == "csr":
            for i in range(n):
                for k in range(t.rowptr[i], t.rowptr[i + 1]):
                    Q[i, t.colidx[k]] += t.vals[k]
        elif t.kind == "dia":
            for k, o in enumerate(t.offsets):
                for i in range(n - o):
                    Q[i, i + o] += t.diags[k][i]
                    if o:
                        Q[i + o, i] += t.diags[k][i]
        elif t.kind in ("factor", "dense_factor"):
            for r in range(t.p):
                row = np.zeros(n)
                if t.kind == "factor":
                    for k in range(t.rowptr[r], t.rowptr[r + 1]):
                        row[t.colidx[k]] += t.vals[k]
                else:
                    row[:] = np.asarray(t.dense).reshape(t.p, n)[r]
                for j1 in range(n):
                    for j2 in range(n):
                        Q[j1, j2] += row[j1] * row[j2]
        else:
            raise ValueError(t.kind)
    return A, Q


def _all_term_kinds(n=11, m=6, seed=5):
    """A QP whose Q sums one term of every stored kind (diagonal, CSR, band with offsets
    0, 1 and 3, sparse factor, dense factor); A with an empty row."""
    rng = np.random.default_rng(seed)
    Ad = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
    Ad[2] = 0.0
    Ad[4, 7] = 3.0
    rp, ci, va = qpgen.csr_from_scipy(sp.csr_matrix(Ad))
    G = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.4)
    S = G + G.T
    srp = [0]; sci = []; sva = []
    for i in range(n):
        for j in range(n):
            if S[i, j] != 0.0:
                sci.append(j); sva.append(S[i, j])
        srp.append(len(sci))
    offs = np.array([0, 1, 3], np.int32)
    diags = rng.uniform(-1, 1, (3, n))
    B = rng.standard_normal((4, n)) * (rng.random((4, n)) < 0.5)
    brp = [0]; bci = []; bva = []
    for r in range(4):
        for j in range(n):
            if B[r, j] != 0.0:
                bci.append(j); bva.append(B[r, j])
        brp.append(len(bci))
    F = rng.standard_normal((3, n))
    terms = [
        qpgen.QTerm("diag", dense=rng.uniform(0.5, 1.5, n)),
        qpgen.QTerm("csr", rowptr=np.array(srp, np.int32), colidx=np.array(sci, np.int32),
                    vals=np.array(sva)),
        qpgen.QTerm("dia", offsets=offs, diags=diags),
        qpgen.QTerm("factor", p=4, rowptr=np.array(brp, np.int32), colidx=np.array(bci, np.int32),
                    vals=np.array(bva)),
        qpgen.QTerm("dense_factor", p=3, dense=np.ascontiguousarray(F)),
    ]
    inf = np.inf
    return qpgen.QP(n, m, rp, ci, va, rng.standard_normal(n), np.full(m, -inf), np.full(m, inf),
                    np.full(n, -inf), np.full(n, inf), 0, 0.0, terms, name="all_term_kinds")


def test_operator_products_of_every_term_kind_match_their_entries():
    """The oracle's Q v, A v and A^T y (the products every step of Algorithm 4 is built from)
    equal the matrices written out entry by entry from each storage form's definition, term
    by term and summed."""
    qp = _all_term_kinds()
    A, Q = _dense_by_entries(qp)
    assert np.allclose(Q, Q.T)
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.standard_normal(qp.n)
        y = rng.standard_normal(qp.m)
        np.testing.assert_allclose(oracle.qmul(qp, v), Q @ v, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(oracle.amul(qp, v), A @ v, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(oracle.atmul(qp, y), A.T @ y, rtol=1e-12, atol=1e-12)
    for t in qp.qterms:
        one = qpgen.QP(**{**qp.__dict__, "qterms": [t]})
        _, Qt = _dense_by_entries(one)
        v = rng.standard_normal(qp.n)
        np.testing.assert_allclose(oracle.qmul(one, v), Qt @ v, rtol=1e-12, atol=1e-12,
                                   err_msg=t.kind)


def _support_by_lp(w, lo, hi):
    """sup over the box [lo, hi] of <w, s>, computed by an LP solver (finite by construction)."""
    if w.size == 0:
        return 0.0
    r = so.linprog(-w, bounds=list(zip(np.where(np.isfinite(lo), lo, None),
                                       np.where(np.isfinite(hi), hi, None))), method="highs")
    assert r.status == 0
    return -r.fun


@pytest.mark.parametrize("phi", ["box", "l1"])
@pytest.mark.parametrize("dominant", ["Ax or Qx", "b", "c", "A*y"])
def test_stopping_measures_at_a_point_away_from_the_solution(phi, dominant):
    """eta_p, eta_d, eta_gap of the Sec. 4.1 stopping rule at an arbitrary (x, y, z): the
    projection onto K and both support functions (delta*_K(-y) = sup_{s in K} <-y, s>,
    phi*(-z) = sup_{x in C} <-z, x> for the box) evaluated by an LP solver, the norms and
    denominators as printed.  y and z carry signs that keep the supports finite, with zero
    multipliers on some infinite bounds (those contribute 0).  Each variant scales one
    quantity so that it is the largest term of its denominator."""
    qp = _all_term_kinds(n=11, m=6, seed=9)
    rng = np.random.default_rng(4)
    n, m = qp.n, qp.m
    qp.l = rng.uniform(-2, 0, m); qp.u = qp.l + rng.uniform(0, 2, m)
    qp.l[[1, 4]] = -np.inf; qp.u[[2, 4]] = np.inf; qp.u[5] = qp.l[5]
    if dominant == "b":
        qp.l[0], qp.u[0] = -400.0, -399.0          # ||b|| = 400 and row 0 violated
    if dominant == "c":
        qp.c = qp.c * 1e3
    y = rng.standard_normal(m) * (1e3 if dominant == "A*y" else 1.0)
    y[~np.isfinite(qp.l)] = -np.abs(y[~np.isfinite(qp.l)])      # y_i > 0 needs l_i finite
    y[~np.isfinite(qp.u)] = np.abs(y[~np.isfinite(qp.u)])       # y_i < 0 needs u_i finite
    y[4] = 0.0                                                   # free row: zero multiplier
    if phi == "box":
        qp.L = rng.uniform(-3, -1, n); qp.U = rng.uniform(1, 3, n)
        qp.L[[0, 6]] = -np.inf; qp.U[[3, 6]] = np.inf
        x = np.clip(rng.standard_normal(n) * 2, qp.L, qp.U)
        z = rng.standard_normal(n)
        z[~np.isfinite(qp.L)] = -np.abs(z[~np.isfinite(qp.L)])
        z[~np.isfinite(qp.U)] = np.abs(z[~np.isfinite(qp.U)])
        z[6] = 0.0
        phi_x = 0.0
        phi_conj = _support_by_lp(-z, qp.L, qp.U)
    else:
        qp.phi = qpgen.PHI_L1; qp.lam = 0.7
        qp.L = np.full(n, -np.inf); qp.U = np.full(n, np.inf)
        x = rng.standard_normal(n)
        z = rng.uniform(-qp.lam, qp.lam, n)                      # phi*(-z) = 0 on |z| <= lambda
        phi_x = qp.lam * np.abs(x).sum()
        phi_conj = 0.0
    A, Q = _dense_by_entries(qp)
    Ax, Qx, Aty = A @ x, Q @ x, A.T @ y
    b = np.maximum(np.where(np.isfinite(qp.l), np.abs(qp.l), 0.0),
                   np.where(np.isfinite(qp.u), np.abs(qp.u), 0.0))
    terms_p = {"b": np.abs(b).max(), "Ax": np.abs(Ax).max()}
    terms_d = {"c": np.abs(qp.c).max(), "A*y": np.abs(Aty).max(), "Qx": np.abs(Qx).max()}
    if dominant in ("b", "c", "A*y"):
        big = terms_p if dominant == "b" else terms_d
        assert max(big, key=big.get) == dominant
    eta_p = np.abs(Ax - np.clip(Ax, qp.l, qp.u)).max() / (1 + max(terms_p.values()))
    eta_d = np.abs(-Qx + Aty + z - qp.c).max() / (1 + max(terms_d.values()))
    supK = _support_by_lp(-y, qp.l, qp.u)
    P = 0.5 * x @ Qx + qp.c @ x + phi_x
    Dv = -0.5 * x @ Qx - supK - phi_conj
    eta_gap = abs(P - Dv) / (1 + max(abs(P), abs(0.5 * x @ Qx + supK + phi_conj)))
    e, pobj, dobj = oracle.eta(qp, x, y, z)
    np.testing.assert_allclose(e, [eta_p, eta_d, eta_gap], rtol=1e-10)
    assert pobj == pytest.approx(P, rel=1e-12) and dobj == pytest.approx(Dv, rel=1e-10)
    assert min(e) > 1e-4                     # a point away from the solution: every term counts


@pytest.mark.parametrize("form", ["csr", "dia"])
def test_scaling_closed_form_when_ruiz_is_already_at_its_fixed_point(form):
    """Q = [[1, 1], [1, 1/4]] (m = 0): every column of K already has infinity norm 1, so the ten
    Ruiz passes leave d = 1, and the Pock-Chambolle pass (alpha = 1) divides by the square roots
    of the column 1-norms 2 and 5/4: d = (1/sqrt 2, 1/sqrt 1.25).  Taking the 1-norm in the Ruiz
    passes, or the infinity norm in the last one, gives another d."""
    Qd = np.array([[1.0, 1.0], [1.0, 0.25]])
    if form == "csr":
        qp = qpgen.from_dense(Qd, np.array([1.0, -1.0]), L=np.array([-1.0, -1.0]), U=np.array([1.0, 1.0]))
    else:
        qp = qpgen.from_dense(None, np.array([1.0, -1.0]), L=np.array([-1.0, -1.0]), U=np.array([1.0, 1.0]))
        qp.qterms = [qpgen.QTerm("dia", offsets=np.array([0, 1], np.int32),
                                 diags=np.array([[1.0, 0.25], [1.0, 0.0]]))]
    d, e, ok = oracle.scaling(qp)
    assert ok and e.size == 0
    np.testing.assert_allclose(d, [1 / np.sqrt(2.0), 1 / np.sqrt(1.25)], rtol=1e-15)


def test_scaling_closed_form_with_one_entry_per_column():
    """K = [Q A^T; A 0] with one nonzero per column (Q diagonal on the columns A does not touch,
    A a scaled partial permutation): the first Ruiz pass makes every entry +-1 and no later pass
    changes it, so d_j = 1/sqrt|q_j| on Q's columns and d_j = e_i = 1/sqrt|a_ij| on A's
    (both start at 1 and are divided by the same root)."""
    n, m = 5, 3
    q = np.array([0.0, 4.0, 0.0, 0.0, 0.09])
    A = np.zeros((m, n))
    A[0, 2], A[1, 0], A[2, 3] = -25.0, 0.01, 2.0
    qp = qpgen.from_dense(np.diag(q), np.ones(n), A=A, l=-np.ones(m), u=np.ones(m),
                          L=-np.ones(n), U=np.ones(n), q_kind="diag")
    d, e, ok = oracle.scaling(qp)
    assert ok
    np.testing.assert_allclose(d, [10.0, 0.5, 0.2, 1 / np.sqrt(2.0), 1 / 0.3], rtol=1e-14)
    np.testing.assert_allclose(e, [0.2, 10.0, 1 / np.sqrt(2.0)], rtol=1e-14)


def test_duplicate_csr_entries_are_summed():
    """A row that stores the same column twice means the sum of the two values (CSR as a list
    of entries): the products equal those of the matrix written out entry by entry."""
    qp = _all_term_kinds(seed=3)
    rp, ci, va = qp.A_rowptr.copy(), qp.A_colidx.copy(), qp.A_vals.copy()
    k = int(rp[1])                                   # append a duplicate of row 0's first entry
    col = int(ci[rp[0]]) if rp[1] > rp[0] else 0
    ci = np.insert(ci, k, col).astype(np.int32)
    va = np.insert(va, k, 0.75)
    rp = rp.copy()
    rp[1:] += 1
    dup = qpgen.QP(**{**qp.__dict__, "A_rowptr": rp, "A_colidx": ci, "A_vals": va})
    A, Q = _dense_by_entries(dup)
    rng = np.random.default_rng(5)
    v, y = rng.standard_normal(dup.n), rng.standard_normal(dup.m)
    np.testing.assert_allclose(oracle.amul(dup, v), A @ v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.atmul(dup, y), A.T @ y, rtol=1e-12, atol=1e-12)
    assert A[0, col] == pytest.approx(_dense_by_entries(qp)[0][0, col] + 0.75)
