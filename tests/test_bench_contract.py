"""Host logic of bench.py that the JSON line rests on (CPU only): workload
defaults, the roofline arithmetic and the DRAM-traffic lookup."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("wl,n,s,pc,prec,restart", [
    ("convdiff3d", 128, 8, "ilu0", "fp32", 30),
    ("convdiff2d", 64, 4, "jacobi", "fp64", 30),
    ("diffreact", 512, 2, "ilu0", "fp32", 64),
    ("richards", 96, 8, "ilu0", "fp32", 64),
])
def test_workload_defaults(wl, n, s, pc, prec, restart):
    a = bench.parse(["--workload", wl])
    assert (a.n, a.s, a.precond, a.precision, a.restart) == (n, s, pc, prec, restart)
    assert bench.linear(a) == wl.startswith("convdiff")
    assert a.steps >= 1 and a.warmup >= 3 and a.gpus == 1


def test_inner_tolerances_follow_the_paper():
    a = bench.parse([])
    assert bench.inner_tol_for(a, 8) == 1e-2            # Sec. 4.1, s > 1
    a = bench.parse(["--workload", "diffreact", "--precision", "fp64"])
    assert bench.inner_tol_for(a, 2) == 1e-5            # Sec. 4.2
    a = bench.parse(["--workload", "richards"])
    assert bench.inner_tol_for(a, 8) == 1e-2


def test_roofline_hbm_and_alu_cases():
    # 10 launches, 1 GB each, 100 us each -> 10 TB/s against a 5 TB/s peak
    prof = {"ms": 1.0, "bytes": 10e9, "flops": 1e6, "launches": 10}
    r = bench.roofline("spmm", prof, 5000.0, "measured", "fp32", "none", 1.3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(10000.0) and r["frac"] == pytest.approx(2.0)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(1e9)
    assert r["avg_launch_us"] == pytest.approx(100.0)
    # float64 with more flop time than byte time: reported against the FP64 rate
    prof = {"ms": 1.0, "bytes": 1e6, "flops": 1e9, "launches": 1}
    r = bench.roofline("gram", prof, 5000.0, "measured", "fp64", "none", 1.25)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # the measured FP64 rate passed in is the denominator
    assert r["achieved"] == pytest.approx(1.0) and r["peak"] == pytest.approx(1.25)
    assert r["frac"] == pytest.approx(0.8)
    assert bench.roofline("x", {"ms": 0.0, "bytes": 0, "flops": 0, "launches": 0}, 1, "m",
                          "fp32", "w", 1.0) is None


def test_traffic_lookup_only_for_the_captured_sources():
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    with open(path) as fh:
        d = json.load(fh)
    for wl, fams in d.items():
        for fam, e in fams.items():
            got = bench.ncu_traffic(fam, wl)
            if e["source_hash"] == bench.source_hash(fam):
                assert got == e["dram_bytes_per_launch"] and got > 0
            else:
                assert got is None
    assert bench.ncu_traffic("ilu", "no-such-workload") is None
    assert bench.ncu_traffic("gram", "convdiff3d_n128_s8_ilu0") is None


def test_source_hash_follows_only_the_family_sources(tmp_path, monkeypatch):
    """A change in another translation unit leaves a family's hash alone; a
    change in one of its own sources changes it."""
    import shutil
    for fam, files in bench.KERNEL_SOURCES.items():
        for rel in files:
            dst = tmp_path / rel
            dst.parent.mkdir(parents=True, exist_ok=True)
            shutil.copy(os.path.join(ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = {f: bench.source_hash(f) for f in bench.KERNEL_SOURCES}
    (tmp_path / "paper_2504_02117_gb300/csrc/krylov.cu").write_text("// another unit\n")
    assert {f: bench.source_hash(f) for f in bench.KERNEL_SOURCES} == before
    with open(tmp_path / "paper_2504_02117_gb300/csrc/ilu.cu", "a") as fh:
        fh.write("// changed\n")
    assert bench.source_hash("ilu") != before["ilu"]
    assert bench.source_hash("spmm") == before["spmm"]


def test_measured_peak_is_read():
    peak, kind = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000.0
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_spbop_byte_model_reduces_to_the_papers_count():
    """Without vector reuse, index bytes or result writes the byte count is
    the paper's (one matrix entry and k vector entries per nonzero, Sec.
    Performance analysis): AI 1/8 for the single vector (the spMV figure of
    Sec. 1) and a gain of about 1.8 at k = 16; the library's own count for
    the 128^3 inner SpMM at s = 8 in float32 is the 259 260 420 bytes its
    profiler recorded for a full-width launch."""
    g = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "spbop_ai.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = float(v)
    paper = dict(idx_bytes=0, vector_reuse=False, write_result=False)
    nnz, n = 14_581_760, 128 ** 3
    assert bench.spbop_ai(nnz, n, 1, **paper) == g["ai_spmv"]
    k = int(g["k"])
    gain = bench.spbop_ai(nnz, n, k, **paper) / bench.spbop_ai(nnz, n, 1, **paper)
    assert g["gain_about"] <= gain < g["gain_about"] + 0.1
    assert abs(bench.spbop_ai(nnz, n, 16, **paper) - 0.2353) < 1e-4
    assert bench.spbop_bytes(nnz, n, 8, val_bytes=4, vec_bytes=4) == 259_260_420
    # with X read once per row the intensity grows with k towards nnz / (n * vec_bytes)
    ai = [bench.spbop_ai(nnz, n, k) for k in (1, 2, 4, 8, 16)]
    assert all(a < b for a, b in zip(ai, ai[1:]))
    assert ai[-1] < 2.0 * nnz / n / (2 * 8)


def test_sweep_summary_ratios():
    rows = [{"precision": "fp32", "s": s, "value": v, "status": 0}
            for s, v in ((1, 1.0), (2, 2.0), (4, 2.5), (8, 3.5), (16, 3.0))]
    rows.append({"precision": "fp64", "s": 1, "value": 2.0, "status": 0})
    rows.append({"precision": "fp64", "s": 8, "value": 1.0, "status": 0})
    sm = bench.sweep_summary(rows)
    assert sm["fp32"] == {"s8_over_s1": 3.5, "best_s": 8, "best_over_s1": 3.5}
    assert sm["fp64"]["s8_over_s1"] == 0.5 and sm["fp64"]["best_s"] == 1


def test_batch_workload_and_solver_options():
    """The batch workload and the batched solver force float64 and Jacobi
    (the batched kernel's method), name their workloads, and default to the
    512-slab mix of the seeded generator."""
    a = bench.parse(["--workload", "batch"])
    assert (a.solver, a.precision, a.precond, a.requests) == ("batch", "fp64", "jacobi", 512)
    assert bench.linear(a)
    b = bench.parse(["--workload", "convdiff2d", "--solver", "batch", "--precision", "fp32",
                     "--precond", "ilu0"])
    assert (b.precision, b.precond) == ("fp64", "jacobi")
    assert bench.solver_label(b).startswith("global GMRES(30)")
    r = bench.parse(["--workload", "richards", "--linearisation", "newton"])
    assert r.linearisation == "newton"
    import synth
    jobs = synth.batch_jobs(7, 512)
    assert len(jobs) == 512 and {j["s"] for j in jobs} == {2, 4, 8, 16}
    assert all(j["dims"][2] == 1 or j["dims"][0] == j["dims"][2] for j in jobs)
    assert synth.batch_jobs(7, 512) == jobs                  # seeded
    assert bench.batch_velocity((16, 16, 16)) == (1.0, 0.5, 0.25)
    assert bench.batch_velocity((32, 32, 1)) == (1.0, 0.5, 0.0)


class _St:
    def __init__(self, status, outer, inner, restarts, rel, flops, ms=2.0):
        self.status, self.outer_its, self.inner_its, self.restarts = status, outer, inner, restarts
        self.col_relres = rel + [0.0] * (16 - len(rel))
        self.flops, self.solve_ms = flops, ms


def test_batch_aggregate_and_float64_roofline():
    """A batch's statistics: worst status and residual, summed steps and
    operations; the roofline divides the kernel's counted float64
    operations by the step time and compares them with the measured rate."""
    agg = bench._AggStats([_St(0, 3, 90, 4, [1e-11, 2e-11], 2e8),
                           _St(4, 5, 30, 2, [3e-9], 1e8)]).as_dict()
    assert agg["status"] == 4 and agg["outer_its"] == 5 and agg["inner_its"] == 120
    assert agg["restarts"] == 6 and agg["flops"] == 3e8 and agg["col_relres"] == [3e-9]
    assert agg["max_inner_its"] == 90
    rl = bench.batch_roofline([agg], 0.5, 1.0)          # 3e8 flops in 0.5 ms
    assert rl["bound"] == "alu" and rl["unit"] == "TFLOP/s"
    assert rl["achieved"] == pytest.approx(0.6) and rl["frac"] == pytest.approx(0.6)
    assert bench.batch_roofline([{"flops": 0.0}], 0.5, 1.0) is None
