#!/usr/bin/env python
"""Benchmark of the vectorised parallel-in-time block solve on GB300.

Metric: time-step*DOF/s of a whole linear time slab (s implicit-Euler steps of
3-D convection-diffusion on 128^3 cells, log-normal diffusion, coupled as one
matrix equation and solved to tol 1e-10 by defect correction around block
GMRES(30) + ILU(0)), plus the achieved HBM bandwidth of the block SpMM and of
the dominant kernel against the measured peak.

A step is one full slab solve (every kernel family of the path: coupled
residual, column norms, inner SpMM, ILU(0) sweeps, block Gram / update,
CholQR2, Hessenberg least squares, outer update), inputs resident in HBM.
`e2e` repeats it through the C ABI from pinned HOST buffers with the B upload
and the Y download inside the timed region.

--impl reference times the CPU oracle on a bounded sample of the same
workload (the oracle is the reference of this build).
Multi-GPU: the path has no data-parallel split of one slab; --gpus N runs N
independent replicas (one slab per GPU), weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("time-step·DOF/s and block-SpMM HBM GB/s (% roofline) at s=1..16, "
          "mixed vs FP64")
UNIT = "time-step*DOF/s"
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 (non-tensor and tensor alike)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="pint", choices=["pint", "reference"])
    p.add_argument("--n", type=int, default=128, help="cells per direction")
    p.add_argument("--s", type=int, default=8, help="coupled time steps (block width)")
    p.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    p.add_argument("--precond", default="ilu0", choices=["ilu0", "jacobi"])
    p.add_argument("--inner-tol", type=float, default=None)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="also time one solve per (s, precision) for s=1..16")
    p.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    return p.parse_args()


def inner_tol_for(args, s):
    if args.inner_tol is not None:
        return args.inner_tol
    if s > 1:
        return 1e-2                       # Sec. 4.1: loose inner solves for s > 1
    return 1e-10 if args.precision == "fp64" else 1e-5


# ----------------------------------------------------------------- oracle
def oracle_sample(n, s, reps=1):
    """Time the oracle's slab solve on an n^3 sample of the workload (this
    process runs with single-threaded BLAS)."""
    import numpy as np
    import synth
    from oracle import coupling, fv, slab
    w = synth.convdiff_3d(n, s)
    D = synth.diffusion_field(w)
    K = fv.convdiff_matrix(w.dims, D, w.velocity)
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, w.tau)
    B = synth.rhs_block(w)
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        slab.slab_solve(K, np.ones(w.n), A1, A2, B, None, tol=w.tol,
                        inner_tol=1e-2 if s > 1 else 1e-10, precond="ilu0")
        times.append(time.perf_counter() - t)
    return {"n": w.n, "s": s, "times": times}


def run_oracle_subprocess(n, s, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n),
                        "--s", str(s), "--steps", str(reps)],
                       capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_02117_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(family, workload):
    """dram bytes per launch of `family` from the committed ncu summary, or
    None when absent or taken from different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(workload, {}).get(family)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def roofline(fam, prof, hbm_peak, peak_kind, precision, workload):
    tot_ms = prof["ms"]
    if tot_ms <= 0 or prof["launches"] == 0:
        return None
    per_launch_s = tot_ms / 1e3 / prof["launches"]
    bytes_pl = prof["bytes"] / prof["launches"]
    flops_pl = prof["flops"] / prof["launches"]
    gbs = bytes_pl / per_launch_s / 1e9
    t_mem = bytes_pl / (hbm_peak * 1e9)
    t_alu = flops_pl / (FP64_PEAK_TFLOPS * 1e12) if precision == "fp64" else 0.0
    if t_alu > t_mem:
        ach = flops_pl / per_launch_s / 1e12
        return {"kernel": fam, "bound": "alu", "achieved": round(ach, 4),
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                "peak_source": "nominal FP64 of GB300 (recipe table)",
                "traffic": ncu_traffic(fam, workload),
                "algorithmic_bytes_per_launch": bytes_pl, "launches": prof["launches"],
                "avg_launch_us": per_launch_s * 1e6}
    return {"kernel": fam, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "traffic": ncu_traffic(fam, workload), "algorithmic_bytes_per_launch": bytes_pl,
            "launches": prof["launches"], "avg_launch_us": per_launch_s * 1e6}


# ------------------------------------------------------------------ main
def main():
    args = parse()
    if args.oracle_sample:
        r = oracle_sample(args.oracle_sample, args.s, max(1, args.steps))
        print(json.dumps(r))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl_name = f"convdiff3d_{args.n}^3_lognormal_s{args.s}_implicit-euler_{args.precond}"

    if args.impl == "reference":
        if rank != 0:
            return
        return reference_arm(args, wl_name, world)

    # CPU baseline first: a spawned single-threaded process, before any GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            samp = 48
            r = run_oracle_subprocess(samp, args.s, 1)
            v = r["s"] * r["n"] / min(r["times"])
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"one full oracle slab solve (FP64, ILU(0), same recipe) on "
                             f"{samp}^3 = {r['n']} cells, s={args.s}: {min(r['times']):.1f} s"}
        except Exception as e:          # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"failed: {e}"[:300]}

    import numpy as np
    import torch
    import synth
    import paper_2504_02117_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = synth.convdiff_3d(args.n, args.s)
    D = synth.diffusion_field(w).ravel()
    B = synth.rhs_block(w)
    n, s = w.n, args.s
    ctx = P.pint_create(local)
    op = P.pint_fv_convdiff(ctx, *w.dims, D, w.velocity)
    A1 = (np.eye(s) - np.eye(s, k=-1)) / w.tau          # implicit Euler, Eq. multistep
    A2 = np.eye(s)
    P.pint_set_coupling(ctx, op, A1, A2)
    prec = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}[args.precision]
    o = P.pint_opts_default()
    o.tol = w.tol
    o.inner_tol = inner_tol_for(args, s)
    o.precond = P.PINT_PC_ILU0 if args.precond == "ilu0" else P.PINT_PC_JACOBI
    o.precision = prec
    Bd = torch.tensor(B, device="cuda", dtype=torch.float64)
    Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream()

    # setup (ILU factorisation happens on the first solve): untimed
    t0 = time.perf_counter()
    st0 = P.pint_solve_block(ctx, op, Bd, None, Y, o)
    setup_solve_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        Y.zero_()
        P.pint_solve_block(ctx, op, Bd, None, Y, o)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    P.pint_profile_reset(ctx)
    P.pint_profile_enable(ctx, True)
    l0 = P.pint_kernel_launches(ctx)
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            Y.zero_()
            st = P.pint_solve_block(ctx, op, Bd, None, Y, o)
            stats.append(st.as_dict(s))
        ev1.record(stream)
        barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = P.pint_kernel_launches(ctx) - l0
    P.pint_profile_enable(ctx, False)
    fams = {name: P.pint_profile_read(ctx, k) for k, name in enumerate(P.KERNEL_FAMILIES)}
    if dist is not None:
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = world * args.steps * s * n / (elapsed_ms / 1e3)

    # correctness of the timed result: residual relative to F (device check)
    relres = max(max(st["col_relres"]) for st in stats)
    converged = all(st["status"] == 0 for st in stats)

    # ------------------------------------------------------------- e2e leg
    e2e = None
    if not args.no_e2e:
        Bh = torch.tensor(B, dtype=torch.float64).pin_memory()
        Yh = torch.empty(n, s, dtype=torch.float64).pin_memory()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            Bd.copy_(Bh, non_blocking=True)
            Y.zero_()
            P.pint_solve_block(ctx, op, Bd, None, Y, o)
            Yh.copy_(Y, non_blocking=True)
        e1.record(stream)
        barrier()
        e_ms = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": world * args.steps * s * n / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(Bh.numel() * 8), "d2h_bytes_per_step": int(Yh.numel() * 8),
               "ms_per_step": e_ms / args.steps}

    if rank != 0:
        P.pint_operator_destroy(op)
        P.pint_destroy(ctx)
        if dist is not None:
            dist.destroy_process_group()
        return

    hbm_peak, peak_kind = measured_peaks()
    total_prof = sum(f["ms"] for f in fams.values()) or 1.0
    dominant = max((k for k in fams if k not in ("vec",)), key=lambda k: fams[k]["ms"])
    kernels = {}
    for k, f in fams.items():
        if f["launches"]:
            kernels[k] = {"launches": f["launches"], "ms": round(f["ms"], 3),
                          "share": round(f["ms"] / total_prof, 4),
                          "GB/s": round(f["bytes"] / max(f["ms"], 1e-9) / 1e6, 1)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else f"f64+{args.precision}",
        "data": "synthetic",
        "config": {"workload": wl_name, "cells": n, "s": s, "nnz": int(P.pint_operator_nnz(op)),
                   "tau": w.tau, "tol": w.tol, "inner_tol": o.inner_tol, "restart": o.restart,
                   "precision": args.precision, "precond": args.precond,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (matrix and basis >> 129 MB), no flush"},
        "roofline": roofline(dominant, fams[dominant], hbm_peak, peak_kind, args.precision,
                             wl_name),
        "spmm_roofline": roofline("spmm", fams["spmm"], hbm_peak, peak_kind, args.precision,
                                  wl_name),
        "kernels": kernels,
        "iterations": {"outer": stats[-1]["outer_its"], "inner": stats[-1]["inner_its"],
                       "restarts": stats[-1]["restarts"]},
        "converged": converged, "max_col_relres": relres,
        "setup": {"first_solve_s": setup_solve_s, "ilu_setup_ms": st0.setup_ms},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(), "impl": "pint",
    }
    if args.sweep:
        out["sweep"] = sweep(P, ctx, args, w)
    print(json.dumps(out), flush=True)
    P.pint_operator_destroy(op)
    P.pint_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def sweep(P, ctx, args, w0):
    """One timed solve per (precision, s) on the same grid (after one warm-up
    solve each): time-step*DOF/s and SpMM GB/s."""
    import numpy as np
    import torch
    import synth
    res = []
    D = synth.diffusion_field(w0).ravel()
    for prec_name in ("fp64", "fp32"):
        for s in (1, 2, 4, 8, 16):
            w = synth.convdiff_3d(args.n, s)
            op = P.pint_fv_convdiff(ctx, *w.dims, D, w.velocity)
            P.pint_set_coupling(ctx, op, (np.eye(s) - np.eye(s, k=-1)) / w.tau, np.eye(s))
            o = P.pint_opts_default()
            o.tol = w.tol
            ns = argparse.Namespace(inner_tol=args.inner_tol, precision=prec_name)
            o.inner_tol = inner_tol_for(ns, s)
            o.precond = P.PINT_PC_ILU0
            o.precision = P.PINT_FP64 if prec_name == "fp64" else P.PINT_FP32
            Bd = torch.tensor(synth.rhs_block(w), device="cuda", dtype=torch.float64)
            Y = torch.zeros(w.n, s, device="cuda", dtype=torch.float64)
            P.pint_solve_block(ctx, op, Bd, None, Y, o)
            Y.zero_()
            P.pint_profile_reset(ctx)
            P.pint_profile_enable(ctx, True)
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = P.pint_solve_block(ctx, op, Bd, None, Y, o)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            P.pint_profile_enable(ctx, False)
            sp = P.pint_profile_read(ctx, 1)
            res.append({"precision": prec_name, "s": s, "value": s * w.n / dt,
                        "solve_s": dt, "outer": st.outer_its, "inner": st.inner_its,
                        "status": st.status,
                        "spmm_GBs": sp["bytes"] / max(sp["ms"], 1e-9) / 1e6})
            P.pint_operator_destroy(op)
            del Bd, Y
    return res


def reference_arm(args, wl_name, world):
    """The oracle as it stands, timed on this host's cores, on a bounded
    sample of the workload per step."""
    samp = 32
    r = run_oracle_subprocess(samp, args.s, args.warmup + args.steps)
    times = r["times"][args.warmup:]
    per = statistics.mean(times)
    v = r["s"] * r["n"] / per
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl_name, "sample_cells": r["n"], "s": args.s},
           "impl": "reference",
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"oracle slab solve on {samp}^3 cells per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
