"""Host-side pieces of bench.py (no GPU): the algorithmic byte / FP64 counts behind the
roofline, and the source hash that keeps a recorded DRAM-traffic table tied to the kernel
code it was measured on."""
import os
import shutil

import numpy as np
import pytest

import bench
import qpgen


def test_tiled_factor_counts():
    """Lasso-like problem (no A, Q = B^T B): the tiled pre-pass group reads B and B^T at 10 B
    per entry, x once, the kb partial rows twice (written and read), t, and u once per tile of
    t plus its re-reads; FP64: two FMAs per entry, the partial sums and the tile updates of u."""
    qp = qpgen.lasso(p=30_000, q=60_000, density=5e-4, seed=2)
    n = qp.n
    t = [q for q in qp.qterms if q.kind == "factor"][0]
    nnz, p = int(t.rowptr[-1]), t.p
    kb, kt = -(-n // 25600), -(-p // 25600)
    assert (kb, kt) == (3, 2)
    b, f = bench.algorithmic(qp, tiled=True)["pre1"]
    assert b == 20 * nnz + 8 * n + 16 * kb * p + 8 * p + 8 * n * (2 * kt - 1)
    assert f == 2 * nnz + kb * p + (kt - 1) * n
    # the row pass then only adds u; untiled it carries the B^T pass (entries, and adding the
    # term to each row: one FP64 operation per row either way)
    bq, fq = bench.algorithmic(qp, tiled=True)["q1"]
    bu, fu = bench.algorithmic(qp, tiled=False)["q1"]
    assert bu - bq == 12 * nnz + 4 * n - 8 * n and fu - fq == nnz + n


def test_zx_counts_match_the_eighteen_operations_per_coordinate():
    # reads x, w, Qw, A^*y with their anchors and bar values, c, L, U; writes x, w, Qw, A^*y,
    # xbar, what, wbar_{1/2}
    qp = qpgen.large_cqp(n=10_000, m=5_000, seed=0)
    b, f = bench.algorithmic(qp)["zx"]
    assert f == 18 * qp.n and b == 8 * qp.n * (15 + 7)


def test_fused_pass_counts():
    # ath: A^T ybar (12 B/entry, 4 B/row, ybar gathered once), 5 n-vector reads and 2 writes;
    # q2h: the Q pass plus 7 reads and 3 writes, 8 FP64 operations per coordinate beyond Q
    qp = qpgen.large_cqp(n=10_000, m=5_000, seed=0)
    n, m, nnzA = qp.n, qp.m, int(qp.A_rowptr[-1])
    alg = bench.algorithmic(qp)
    assert alg["ath"] == (12 * nnzA + 4 * n + 8 * m + 8 * n * 7, nnzA + 8 * n)
    bq, fq = alg["q2"]
    bh, fh = alg["q2h"]
    assert bh - bq == 8 * n * 8 and fh - fq == 8 * n


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2507_02470_gb300", "csrc")
    dst = tmp_path / "paper_2507_02470_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.STEP_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_sha()
    k = dst / "kernels.cuh"
    k.write_text(k.read_text() + "\n// a comment added at the end\n\n")
    assert bench.source_sha() == h0
    k.write_text(k.read_text() + "static int added_code = 1;\n")
    assert bench.source_sha() != h0


def test_roofline_takes_the_slowest_kernel_and_the_larger_fraction():
    """The roofline object: the kernel with the largest mean time, achieved = algorithmic count
    / time, frac against the measured HBM copy rate or the FP64 issue peak (the probe's lanes
    per clock x SMs x the maximum clock, passed in), whichever fraction is larger, and that
    kernel's recorded DRAM traffic; the whole iteration by the hot-path byte count."""
    qp = qpgen.large_cqp(n=10_000, m=5_000, seed=0)
    alg = bench.algorithmic(qp)
    pk = {"hbm_gbs": 6786.2, "sm_max_mhz": 2070.0}
    fp64_peak = 152 * 1.6817 * 2070e6 / 1e9
    fp64 = (fp64_peak, 1.6817, "probe")
    prof = {"zx": 0.0005, "q1": 0.0004, "a1": 0.0002, "at": 0.0003, "q2": 0.0003, "pre1": 0.0001,
            "pre2": 0.0001, "restart": 0.0}
    r = bench.roofline(prof, qp, pk, "measured", {"zx": 1.5e6, "q1": 2.0e6}, iter_s=2e-6, fp64=fp64)
    assert r["kernel"] == "zx" and r["traffic"] == 1.5e6
    b, f = alg["zx"]
    gbs, ops = b / 0.5e-6 / 1e9, f / 0.5e-6 / 1e9
    assert r["alg_bytes"] == b and r["alg_fp64"] == f
    if ops / fp64_peak > gbs / 6786.2:
        assert r["bound"] == "alu" and r["frac"] == pytest.approx(ops / fp64_peak, abs=1e-4)
        assert r["hbm_frac"] == pytest.approx(gbs / 6786.2, abs=1e-4)
    else:
        assert r["bound"] == "hbm" and r["frac"] == pytest.approx(gbs / 6786.2, abs=1e-4)
    ib = bench.iteration_bytes(qp)
    assert r["iteration"]["alg_bytes"] == ib
    assert r["iteration"]["hbm_frac"] == pytest.approx(ib / 2e-6 / 1e9 / 6786.2, abs=1e-4)
    # a slower row pass takes over the line; the HBM bound wins when its fraction is larger
    prof["a1"] = 0.01
    r = bench.roofline(prof, qp, pk, "measured", None, fp64=fp64)
    assert r["kernel"] == "a1" and r["traffic"] is None and "iteration" not in r
    b, f = alg["a1"]
    assert (r["bound"] == "hbm") == (b / 1e-5 / 1e9 / 6786.2 >= f / 1e-5 / 1e9 / fp64_peak)


def test_iteration_bytes_of_the_large_cqp():
    """The per-iteration byte count of the n = 1e6, m = 5e5 CQP: A and A^T (3e6 entries each at
    12 B), Q twice (three stored diagonals, S and S^T with 3e4 entries), row pointers at 4 B,
    26 n-vector and 8 m-vector passes: about 0.38 GB."""
    qp = qpgen.large_cqp(n=1_000_000, m=500_000, seed=0)
    n, m = 1_000_000, 500_000
    q = 8 * 3 * n + 24 * 30_000 + 4 * (10_000 + 1)
    expect = 24 * 3_000_000 + 2 * q + 4 * (2 * m + 2 * n) + 8 * (26 * n + 8 * m)
    assert bench.iteration_bytes(qp) == expect
    assert 0.37e9 < expect < 0.40e9


def test_clock_summary_median_and_throttle_reasons():
    """nvidia-smi rows (index, SM MHz, max SM MHz, power, active mask, hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap): the median SM clock, the maximum,
    and the reasons seen Active at least once ('Not Active' is not a reason; '[N/A]' clocks are
    skipped)."""
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]
    na, act = "Not Active", "Active"
    cs.samples = [
        ["0", "2070", "2070", "900.1", "0x0", na, na, na, na],
        ["0", "1980", "2070", "1390.5", "0x4", na, na, na, act],
        ["0", "[N/A]", "2070", "1000.0", "0x0", na, na, na, na],
        ["0", "2010", "2070", "1200.0", "0x0", na, na, na, na],
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    cs.samples.append(["0", "1500", "2070", "1400.0", "0x48", na, act, na, na])
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_l2_note_states_which_timing_rule_applies():
    """The n = 1e6 CQP's working set exceeds the 129 MB L2 (no flush needed); the n = 1e3 CQP's
    fits and the note says it is not flushed because each step is a whole solve."""
    big = bench.working_set_bytes(qpgen.large_cqp(n=1_000_000, m=500_000, seed=0))
    small = bench.working_set_bytes(qpgen.plain_cqp())
    assert big > 129e6 > 1e6 > small
    assert bench.l2_note(big).startswith("inputs larger than L2")
    assert "fits in L2" in bench.l2_note(small) and "whole solve" in bench.l2_note(small)


def test_committed_network_matches_the_learned_configuration():
    """The network that the default line's 'learned' key evaluates: MLP 512-1024-1024-257 for
    the n = 1e5, m = 5e4 family, trained on the configured 20,000 members, weights as BF16 bits,
    the mean training solution over all n + m coordinates."""
    z = np.load(bench.NETWORK)
    assert list(z["dims"]) == [512, 1024, 1024, 257]
    assert int(z["n"]) == 100_000 and int(z["m"]) == 50_000
    assert int(z["meta_train"]) == 20_000 and int(z["meta_epochs"]) == 30
    assert z["mu"].shape == (150_000,) and np.all(np.isfinite(z["mu"]))
    for li, (o, i) in enumerate(((1024, 512), (1024, 1024), (257, 1024))):
        W = (z[f"W{li}"].astype(np.uint32) << 16).view(np.float32)
        assert W.shape == (o, i) and np.all(np.isfinite(W)) and z[f"b{li}"].shape == (o,)
    assert float(z["meta_lambda_A"]) > 0 and float(z["meta_lambda_Q"]) > 0
