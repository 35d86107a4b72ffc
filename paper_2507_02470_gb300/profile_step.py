"""Per-kernel timings of the HPR-QP inner step on one of the synthetic workloads.

    python -m paper_2507_02470_gb300.profile_step --workload c1 --iters 30

Creates the solver with stream launches (launch_mode 2, which external profilers can attach
to kernel by kernel), runs a short solve to fix lambda_A, lambda_Q and sigma, then
``hprqp_profile``: `iters` inner steps launched one kernel at a time with CUDA events around
each.  Prints one JSON line with the mean milliseconds of every kernel kind.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c1", choices=["c0", "c1", "c2", "c4"],
                    help="c0: CQP n=1e3, m=500; c1: CQP n=1e6, m=5e5; c2: Lasso 5e4 x 5e5; "
                         "c4: CQP n=1e5, m=5e4 (the learned warm start's family base)")
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--warm-iters", type=int, default=20, help="iterations of the solve before profiling")
    ap.add_argument("--autotune", type=int, default=1,
                    help="SpMV schedule: 1 timed choice, 0 lanes from row length, 2 staged chunks")
    ap.add_argument("--tiled-factor", type=int, default=1,
                    help="shared-memory-tiled factor products: 1 auto, 0 off, 2 forced")
    ap.add_argument("--factor-inline", type=int, default=1,
                    help="thin factor products formed inside the Q pass: 1 auto, 0 off (pre-pass), 2 forced")
    ap.add_argument("--fused-steps", type=int, default=1,
                    help="plain steps end with the fused passes (1) or run all five passes (0)")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import qpgen
    import paper_2507_02470_gb300 as pkg
    pkg.build()
    qp = {"c0": lambda: qpgen.plain_cqp(),
          "c1": lambda: qpgen.large_cqp(n=1_000_000, m=500_000, seed=0),
          "c2": lambda: qpgen.lasso(),
          "c4": lambda: qpgen.param_family_base(n=100_000, m=50_000, seed=0)}[args.workload]()
    with pkg.Solver(qp, launch_mode=2, autotune=args.autotune, tiled_factor=args.tiled_factor,
                    factor_inline=args.factor_inline, fused_steps=args.fused_steps) as s:
        s.solve(tol=1e-30, max_iter=args.warm_iters)
        k = s.kkt()
        ms = s.profile(iters=args.iters)
    print(json.dumps({"workload": args.workload, "autotune": args.autotune, "tiled_factor": args.tiled_factor,
                      "n": qp.n, "m": qp.m,
                      "iters": args.iters,
                      "lambda_A": k["lambda_A"], "lambda_Q": k["lambda_Q"],
                      "lanes": {q: k["lanes_" + q] for q in ("q", "a", "at", "pre")},
                      "ms": {a: round(b, 5) for a, b in ms.items()}}), flush=True)


if __name__ == "__main__":
    main()
