"""The C-ABI library builds, loads and exports every symbol include/hprqp.h declares (no GPU)."""
import os
import re

import pytest

import paper_2507_02470_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(hprqp_\w+)\s*\(", txt, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.lib()


def test_library_exports_header_symbols(lib):
    declared = _declared()
    assert {"hprqp_create", "hprqp_solve", "hprqp_get", "hprqp_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    from paper_2507_02470_gb300._lib import SIGNATURES
    bound = {s[0] for s in SIGNATURES}
    assert _declared() <= bound


def test_default_params_are_the_paper_values(lib):
    p = pkg.default_params()
    assert (p.alpha1, p.alpha2, p.alpha3, p.alpha3_tight, p.ratio_tight) == (0.2, 0.8, 0.5, 0.2, 0.1)
    assert p.check_every == 100 and p.restart_every == 10
    assert p.power_safety == 1.01 and p.iters_per_launch >= 1


def test_oracle_and_library_share_the_defaults(lib):
    import oracle
    o = oracle.default_params()
    p = pkg.default_params()
    for k in ("check_every", "restart_every", "alpha1", "alpha2", "alpha3", "alpha3_tight", "ratio_tight",
              "power_max_iter", "power_tol", "power_safety", "halpern_total", "sigma_golden", "scaling"):
        assert o[k] == getattr(p, k), k


def test_struct_sizes_match_header(lib):
    # compile a tiny C program against the header and compare sizeof with ctypes
    import ctypes
    import subprocess
    import tempfile
    from paper_2507_02470_gb300._lib import hprqp_kkt, hprqp_params, hprqp_qop, hprqp_qterm
    src = ('#include <stdio.h>\n#include "hprqp.h"\nint main(){printf("%zu %zu %zu %zu\\n", sizeof(hprqp_qterm),'
           ' sizeof(hprqp_qop), sizeof(hprqp_params), sizeof(hprqp_kkt));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    assert [int(v) for v in out] == [ctypes.sizeof(hprqp_qterm), ctypes.sizeof(hprqp_qop),
                                     ctypes.sizeof(hprqp_params), ctypes.sizeof(hprqp_kkt)]


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import qpgen
    qp = qpgen.random_small(n=4, m=2, seed=0)
    with pytest.raises(pkg.HPRQPError):
        pkg.Solver(qp)


@pytest.mark.parametrize("bad", [dict(check_every=0), dict(restart_every=0), dict(iters_per_launch=0),
                                 dict(iters_per_launch=4097), dict(launch_mode=4), dict(method=3)])
def test_out_of_range_parameters_are_rejected_before_any_device_work(lib, bad):
    """Parameter ranges are checked first, so the answer is INVALID_ARG with a message naming
    the ranges, on a machine with or without a GPU."""
    import qpgen
    qp = qpgen.random_small(n=4, m=2, seed=0)
    with pytest.raises(pkg.HPRQPError) as e:
        pkg.Solver(qp, **bad)
    assert e.value.status == 4 and "check_every" in str(e.value)
