"""The CUDA path against iterates computed by hand (tests/golden), independently of the oracle.

One-variable problems (n = 1): Algorithm 4 with fixed sigma and no restarts (eqs. (3.1)-(3.3)
and the Halpern step), and the primal methods of Appendix A (Algorithms 6 and 7).  The hand
values are exact fractions; the GPU forms them with fused multiply-adds, hence 1e-14.
"""
import os

import numpy as np
import pytest

import qpgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_02470_gb300 as p
    p.build()
    return p


def test_algorithm4_hand_computed_iterates(pkg):
    g = _golden("hand_1d_iterates.txt")
    qp = qpgen.from_dense(np.array([[g["q"]]]), np.array([g["c"]]), L=np.array([g["L"]]),
                          U=np.array([g["U"]]), q_kind="diag")
    with pkg.Solver(qp, lambda_A=0.0, lambda_Q=g["lambda_Q"], sigma0=g["sigma"], restart_off=1,
                    sigma_fixed=1, scaling=0) as s:
        for k in range(3):
            s.solve(tol=1e-30, max_iter=k + 1)
            x, _, z, w, kkt = s.get()
            assert kkt["iters"] == k + 1
            assert x[0] == pytest.approx(g[f"xbar{k}"], abs=1e-14), k
            assert z[0] == pytest.approx(g[f"zbar{k}"], abs=1e-14), k
            assert w[0] == pytest.approx(g[f"wbar{k}"], abs=1e-14), k


@pytest.mark.parametrize("method", [1, 2])
def test_primal_methods_hand_computed_iterates(pkg, method):
    g = _golden("hand_1d_primal_iterates.txt")
    qp = qpgen.from_dense(np.array([[g["q"]]]), np.array([g["c"]]), A=np.array([[1.0]]),
                          l=np.array([-np.inf]), u=np.array([g["U_row"]]), L=np.array([g["L"]]),
                          U=np.array([g["U"]]))
    with pkg.Solver(qp, method=method, scaling=0, sigma0=g["sigma"], lambda_A=g["lambda_A"],
                    lambda_Q=g["lambda_Q"]) as s:
        for k in range(3):
            s.solve(tol=1e-30, max_iter=k + 1)
            x, y, _, _, _ = s.get()
            assert x[0] == pytest.approx(g[f"p{method}_xbar{k}"], abs=1e-14), k
            assert y[0] == pytest.approx(g[f"p{method}_ybar{k}"], abs=1e-14), k
