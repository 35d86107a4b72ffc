"""The allocation-free power method (hprqp_power_noalloc) through the C ABI.

hprqp_power_noalloc serves callers that cannot allocate device memory when they need
lambda_A: a real-time loop that must not allocate after start-up, or a process whose device
memory belongs to another framework's allocator.  It keeps its scratch in a fixed device array
that every call shares, so two calls in a row must each give the estimate that the CPU oracle's
power method gives (same start vector, Rayleigh quotient and stopping rule), which lies within
the safety factor above the dense lambda_1(A A^T), and the estimate of the solver's own entry
point (hprqp_solve, which runs the same power method in memory it allocated).  This file is
collected last on purpose: the test must pass alone in a fresh process and after all the others.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import qpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def _device_csr(torch, M):
    M = sp.csr_matrix(M)
    return (torch.from_numpy(M.indptr.astype(np.int32)).cuda(), torch.from_numpy(M.indices.astype(np.int32)).cuda(),
            torch.from_numpy(M.data.astype(np.float64)).cuda())


def _call(pkg, torch, qp, max_iter, tol, safety, stream):
    A = qp.A_scipy()
    a_rp, a_ci, a_v = _device_csr(torch, A)
    t_rp, t_ci, t_v = _device_csr(torch, A.T.tocsr())
    lam = C.c_double(0.0)
    st = pkg.lib().hprqp_power_noalloc(qp.m, qp.n, a_rp.data_ptr(), a_ci.data_ptr(), a_v.data_ptr(),
                                       t_rp.data_ptr(), t_ci.data_ptr(), t_v.data_ptr(), max_iter, tol, safety,
                                       stream.cuda_stream, C.byref(lam))
    return st, lam.value


@pytest.mark.parametrize("n,m", [(300, 150), (20000, 10000)])
def test_power_noalloc_matches_oracle_and_solver(pkg, n, m):
    torch = pytest.importorskip("torch")
    qp = qpgen.large_cqp(n=n, m=m, seed=2) if n > 1000 else qpgen.plain_cqp(n=n, m=m, seed=1, q_rows=30,
                                                                             a_density=0.05, q_density=0.1)
    p = pkg.default_params()
    max_iter, tol, safety = int(p.power_max_iter), float(p.power_tol), float(p.power_safety)
    ref = oracle.power_A(qp, max_iter, tol, safety)
    with pkg.Solver(qp, scaling=0) as s:     # the unscaled A, as passed to the no-alloc call
        s.solve(tol=1e-30, max_iter=1)
        solver_lam = s.kkt()["lambda_A"]
    la = None
    if n <= 1000:
        A = qp.A_scipy().toarray()
        la = np.linalg.eigvalsh(A @ A.T).max()
    stream = torch.cuda.Stream()
    for _ in range(2):  # two calls in a row share the same scratch array
        st, lam = _call(pkg, torch, qp, max_iter, tol, safety, stream)
        assert st == 0
        # the same iteration in another summation order: the stopping rule (relative change <=
        # tol) may end the two one step apart, which moves the estimate by less than tol
        assert abs(lam - ref) <= 10 * tol * ref, (lam, ref)
        assert abs(lam - solver_lam) <= 10 * tol * solver_lam, (lam, solver_lam)
        if la is not None:
            assert la <= lam <= safety * la * (1 + 1e-9), (lam, la)


def test_power_noalloc_with_the_largest_iteration_limit(pkg):
    """max_iter = 2^63 - 1: the launch rounds are counted without overflow and the call stops
    at the power method's own stopping rule."""
    torch = pytest.importorskip("torch")
    qp = qpgen.plain_cqp(n=300, m=150, seed=1, q_rows=30, a_density=0.05, q_density=0.1)
    stream = torch.cuda.Stream()
    st0, lam0 = _call(pkg, torch, qp, 5000, 1e-6, 1.01, stream)
    st1, lam1 = _call(pkg, torch, qp, (1 << 63) - 1, 1e-6, 1.01, stream)
    assert st0 == 0 and st1 == 0 and lam1 == lam0 and lam0 > 0


def test_power_noalloc_rejects_oversize(pkg):
    L = pkg.lib()
    lam = C.c_double(0.0)
    too_big = (1 << 17) + 1
    st = L.hprqp_power_noalloc(too_big, 10, 1, 1, 1, 1, 1, 1, 10, 1e-6, 1.01, None, C.byref(lam))
    assert st == 4  # HPRQP_INVALID_ARG, returned before any device access
