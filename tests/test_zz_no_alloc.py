"""The allocation-free power method (hprqp_power_noalloc) against the solver's own estimate.

hprqp_power_noalloc serves callers that cannot allocate device memory when they need
lambda_A (inside a stream capture, in a real-time loop, or under another framework's
allocator).  It keeps its scratch in a fixed device array, so two calls in a row must give
the same estimate as hprqp_solve, which runs the same power method with memory it allocated
itself.  This file is collected last on purpose: the test must pass alone in a fresh process
and after all the others.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

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


@pytest.mark.parametrize("n,m", [(300, 150), (20000, 10000)])
def test_power_noalloc_matches_solver(pkg, n, m):
    torch = pytest.importorskip("torch")
    qp = qpgen.large_cqp(n=n, m=m, seed=2) if n > 1000 else qpgen.plain_cqp(n=n, m=m, seed=1, q_rows=30,
                                                                             a_density=0.05, q_density=0.1)
    with pkg.Solver(qp) as s:
        s.solve(tol=1e-30, max_iter=1)
        ref = s.kkt()["lambda_A"]
        p = s.params
        max_iter, tol, safety = int(p.power_max_iter), float(p.power_tol), float(p.power_safety)
    A = qp.A_scipy()
    a_rp, a_ci, a_v = _device_csr(torch, A)
    t_rp, t_ci, t_v = _device_csr(torch, A.T.tocsr())
    L = pkg.lib()
    stream = torch.cuda.Stream()
    for _ in range(2):  # two calls in a row share the same scratch array
        lam = C.c_double(0.0)
        st = L.hprqp_power_noalloc(m, n, a_rp.data_ptr(), a_ci.data_ptr(), a_v.data_ptr(), t_rp.data_ptr(),
                                   t_ci.data_ptr(), t_v.data_ptr(), max_iter, tol, safety, stream.cuda_stream,
                                   C.byref(lam))
        assert st == 0
        # both run the same iteration; the stopping rule (relative change <= power_tol) may
        # end them one step apart when the row sums round differently, which moves the
        # Rayleigh quotient by less than power_tol relative
        assert abs(lam.value - ref) <= tol * ref, (lam.value, ref)


def test_power_noalloc_rejects_oversize(pkg):
    L = pkg.lib()
    lam = C.c_double(0.0)
    too_big = (1 << 17) + 1
    st = L.hprqp_power_noalloc(too_big, 10, 1, 1, 1, 1, 1, 1, 10, 1e-6, 1.01, None, C.byref(lam))
    assert st == 4  # HPRQP_INVALID_ARG, returned before any device access
