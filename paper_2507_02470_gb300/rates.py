"""Measured arithmetic issue rates of the current GPU (the FP64 roof of this library).

    python -m paper_2507_02470_gb300.rates

Runs ``hprqp_fp64_rate`` for FP64 FMA, add and multiply with all 32 lanes and with 16 lanes
of each warp active, and FP32 FMA for comparison, and prints one JSON line: per operation the
thread operations per SM clock per SM, the SM clock seen and the device-wide rate.  The FP64
FMA figure with full warps, times the SM count and the maximum SM clock, is the FP64 peak
against which ``bench.py`` states the kernels' FP64 fractions.
"""
from __future__ import annotations

import json
import os
import sys


def measure(repeats: int = 3):
    import paper_2507_02470_gb300 as pkg

    names = {0: "dfma", 1: "dadd", 2: "dmul", 3: "ffma"}
    out = {}
    for op, name in names.items():
        for lanes in (32, 16):
            if op == 3 and lanes == 16:
                continue
            best = None
            for _ in range(repeats):
                r = pkg.fp64_rate(op, lanes)
                if best is None or r["lanes_per_clk"] > best["lanes_per_clk"]:
                    best = r
            out[f"{name}_x{lanes}"] = {k: round(v, 4) if k != "ops_per_s" else float(f"{v:.4g}")
                                      for k, v in best.items()}
    return out


def main():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    import paper_2507_02470_gb300 as pkg
    pkg.build()
    torch.cuda.init()
    props = torch.cuda.get_device_properties(0)
    res = measure()
    res["device"] = props.name
    res["sms"] = props.multi_processor_count
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
