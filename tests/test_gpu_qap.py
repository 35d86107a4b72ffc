"""The QAP-relaxation operator of Sec. 4.5 (a matrix-free Q term applied by the library's FP64
contraction kernels) against the oracle: operator products, power method, first iterates in every launch mode that
supports it, and the converged objective."""
import numpy as np
import pytest

import oracle
import qpgen
from tests import dense_ref as D
from tests.parity import close  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


@pytest.fixture(scope="module")
def qaps():
    return {d: qpgen.qap_relaxation(d=d, seed=d) for d in (8, 12)}


def test_qap_operator_and_power_method(pkg, qaps):
    qp = qaps[12]
    _, Q = D.dense_of(qp)
    v = np.random.default_rng(0).standard_normal(qp.n)
    with pkg.Solver(qp) as s:
        assert np.allclose(s.apply("Q", v), Q @ v, rtol=1e-12, atol=1e-10 * np.abs(Q).max())
        s.solve(tol=1e-30, max_iter=1)
        lq = s.kkt()["lambda_Q"]
    top = np.linalg.eigvalsh(Q).max()
    assert top <= lq <= 1.01 * top * (1 + 1e-5)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("d", [8, 12])
def test_qap_first_iterates(pkg, qaps, d, mode):
    qp = qaps[d]
    K = 50
    ref = oracle.solve(qp, tol=1e-30, max_iter=K, trace_len=K)
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q, launch_mode=mode) as s:
        for k in (1, 2, 11, 21, 50):
            s.solve(tol=1e-30, max_iter=k)
            x, y, *_ = s.get()
            assert close(x, ref.trace["x"][k - 1]) <= 1e-10, k
            assert close(y, ref.trace["y"][k - 1]) <= 1e-10, k


def test_qap_converged_objective(pkg, qaps):
    qp = qaps[12]
    ref = oracle.solve(qp, tol=1e-8, max_iter=400000)
    assert ref.status == "converged"
    with pkg.Solver(qp, lambda_A=ref.lambda_A, lambda_Q=ref.lambda_Q) as s:
        assert s.solve(tol=1e-8, max_iter=400000) == "converged"
        x, y, z, w, k = s.get()
    assert abs(k["pobj"] - ref.pobj) <= 1e-6 * (1 + abs(ref.pobj))
    e, _, _ = oracle.eta(qp, x, y, z)
    assert np.max(e) <= 1.05e-8
    X = x.reshape(12, 12, order="F")
    assert np.allclose(X.sum(axis=0), 1, atol=1e-6) and np.allclose(X.sum(axis=1), 1, atol=1e-6)


def test_qap_rejects_persistent_mode(pkg, qaps):
    from paper_2507_02470_gb300 import HPRQPError
    with pytest.raises(HPRQPError):
        pkg.Solver(qaps[8], launch_mode=3)


@pytest.mark.parametrize("d", [50, 200])
def test_qap_contraction_kernels_match_oracle(pkg, d):
    """The hand-written FP64 contractions (Ahat X, then [T1 | S | X][Bhat; -X; -T]) on sizes
    with ragged 32 x 32 tiles (d = 50) and with the K range split across blocks (d = 200: three
    splits summed by the last block of each tile): the operator against the oracle's, element
    by element, and bit-identical on a second application (fixed summation order)."""
    qp = qpgen.qap_relaxation(d=d, seed=d)
    v = np.random.default_rng(d).standard_normal(qp.n)
    ref = oracle.qmul(qp, v)
    with pkg.Solver(qp) as s:
        out = s.apply("Q", v)
        again = s.apply("Q", v)
    assert close(out, ref) <= 1e-13, close(out, ref)
    assert np.array_equal(out, again)
