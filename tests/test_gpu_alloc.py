"""Library-owned device memory through PyTorch's caching allocator (the boundary's ownership
rule): hprqp_create copies every input into memory the handle owns, obtained through the
allocator hooks of hprqp_params, which the Python binding points at torch's caching allocator
by default.  With the hooks no device byte of the handle comes from cudaMalloc; the solve
matches the oracle; torch sees the handle's memory while it lives and gets it back after.
torch_alloc=False takes the library's own cudaMalloc path (the C default) with the same result.
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


def test_solver_memory_comes_from_the_torch_caching_allocator(pkg):
    torch = pytest.importorskip("torch")
    qp = qpgen.plain_cqp(n=300, m=150, seed=3, q_rows=30, a_density=0.05, q_density=0.1)
    ref = oracle.solve(qp, tol=1e-8, max_iter=200000)
    trace = oracle.solve(qp, tol=1e-30, max_iter=40, trace_len=40, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:   # default: torch allocator
        ms = s.memory_stats()
        assert ms["cudamalloc_allocs"] == 0 and ms["cudamalloc_bytes"] == 0, ms
        assert ms["hook_allocs"] > 0 and s._alloc.count == ms["hook_allocs"]
        assert torch.cuda.memory_allocated() - before >= ms["hook_bytes"]
        s.solve(tol=1e-30, max_iter=40)
        x, y, *_ = s.get()
        assert close(x, trace.trace["x"][39]) <= 1e-10 and close(y, trace.trace["y"][39]) <= 1e-10
        assert s.solve(tol=1e-8, max_iter=200000) == "converged"
        k = s.kkt()
        assert abs(k["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))
        assert s.memory_stats()["cudamalloc_allocs"] == 0   # nothing allocated behind the hooks later
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    with pkg.Solver(qp, torch_alloc=False, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        ms = s.memory_stats()
        assert ms["hook_allocs"] == 0 and ms["cudamalloc_allocs"] > 0
        assert s.solve(tol=1e-8, max_iter=200000) == "converged"
        assert abs(s.kkt()["pobj"] - k["pobj"]) <= 1e-12 * (1 + abs(k["pobj"]))


def test_batch_memory_comes_from_the_torch_caching_allocator(pkg):
    torch = pytest.importorskip("torch")
    probs = [qpgen.portfolio(s, n=n) for s, n in ((31, 120), (32, 400))]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with pkg.BatchSolver(probs) as b:
        assert b._alloc is not None and b._alloc.count > 0
        assert torch.cuda.memory_allocated() > before
        assert b.solve(tol=1e-8, max_iter=400000) == "converged"
        for i, qp in enumerate(probs):
            ref = oracle.solve(qp, tol=1e-8, max_iter=400000, scaling=0)
            assert abs(b.get(i)[3]["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
