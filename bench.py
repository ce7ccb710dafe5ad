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
FP64_NOMINAL_TFLOPS = 1.25   # nominal GB300 FP64 (context; the rooflines use the measured rate)


WORKLOADS = {
    # name: (cells per direction, s, precond, precision, description)
    "convdiff3d": (128, 8, "ilu0", "fp32",
                   "3-D conv.-diffusion {n}^3, log-normal D (sigma 1), implicit Euler tau=1e-3, "
                   "slab of s steps, {solver}+{pc}, tol 1e-10"),
    "convdiff2d": (64, 4, "jacobi", "fp64",
                   "2-D conv.-diffusion {n}^2, D=1, v=(1,0.5), implicit Euler tau=1e-3, slab of "
                   "s steps, {solver}+{pc}, tol 1e-10"),
    "diffreact": (512, 2, "ilu0", "fp32",
                  "2-D diffusion-reaction {n}^2, SDIRK2 window of s=2 stages pipelined over 4 "
                  "steps (Algorithm 1), Newton + {solver}+{pc}"),
    "richards": (96, 8, "ilu0", "fp32",
                 "3-D Richards {n}^3, van Genuchten alpha=1 n=2, K_S=exp(2g) correlated 8 "
                 "cells, implicit Euler tau=1/96 window s=8 pipelined over 8 steps, {lin} + "
                 "{solver}+{pc}"),
    "batch": (64, 16, "jacobi", "fp64",
              "batched persistent solve: {requests} slabs in one launch (captured CUDA graph), "
              "2-D 32^2-64^2 and 3-D 16^3-32^3 conv.-diffusion, log-normal D, s in 2..16, "
              "implicit Euler tau=1e-3, {solver}+{pc}, FP64, tol 1e-10"),
    "serve": (128, 16, "ilu0", "fp32",
              "serving: seeded Poisson stream of slab-solve requests (3-D conv.-diffusion, "
              "grids 32^3-{n}^3, s in 2..16, FP32 or FP64 inner solves, {solver}+{pc}, "
              "tol 1e-10), continuous batching over CUDA streams"),
}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="pint", choices=["pint", "reference"])
    p.add_argument("--workload", default="convdiff3d", choices=sorted(WORKLOADS))
    p.add_argument("--n", type=int, default=None, help="cells per direction")
    p.add_argument("--s", type=int, default=None, help="coupled time steps (block width)")
    p.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16"])
    p.add_argument("--precond", default=None, choices=["ilu0", "jacobi"])
    p.add_argument("--inner-tol", type=float, default=None)
    p.add_argument("--restart", type=int, default=None, help="GMRES restart length (30)")
    p.add_argument("--solver", default="gmres",
                   choices=["gmres", "cg", "bicgstab", "global", "batch"],
                   help="inner solver (cg: symmetric systems, e.g. the Richards L-scheme; "
                        "bicgstab: the paper's solver for the linear convection-diffusion "
                        "problem; global: global GMRES on the unsplit operator; batch: the "
                        "same method in the persistent batched kernel, one cluster per slab)")
    p.add_argument("--linearisation", default="lscheme", choices=["lscheme", "newton"],
                   help="richards: the L-scheme of Sec. 4.3 (L = sup theta') or Newton")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-other", action="store_true",
                   help="convdiff3d: skip the compact legs of the other configurations")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-fp64", action="store_true",
                   help="skip the pure-FP64 run of the same workload")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the s = 1..16 sweep (one timed solve per s and precision)")
    p.add_argument("--requests", type=int, default=512,
                   help="serve: requests in the stream; batch: slabs in the launch")
    p.add_argument("--rate", type=float, default=4.0,
                   help="serve: mean arrivals per second (512 requests at 8/s arrive faster "
                        "than one GB300 serves them, about 5.4/s)")
    p.add_argument("--slots", type=int, default=4, help="serve: concurrent solves")
    p.add_argument("--batch-cluster", type=int, default=0,
                   help="batched kernel: CTAs per cluster (0 = the library's choice)")
    p.add_argument("--batch-threads", type=int, default=0,
                   help="batched kernel: threads per CTA (0 = the library's choice)")
    p.add_argument("--no-batch-lane", action="store_true",
                   help="serve: solve the small float64 requests in the slots as well, "
                        "not in batched launches")
    p.add_argument("--batch-max-unknowns", type=int, default=1 << 19,
                   help="serve: largest N*s a float64 request may have for the batch lane")
    p.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    a = p.parse_args(argv)
    dn, ds, dpc, dprec, _ = WORKLOADS[a.workload]
    a.n = a.n or dn
    a.s = a.s or ds
    a.precond = a.precond or dpc
    a.precision = a.precision or dprec
    if a.workload == "batch":
        a.solver = "batch"
    if a.solver in ("global", "batch"):   # the unsplit operator's solvers run in float64
        a.precision = "fp64"
    if a.solver == "batch":               # the batched kernel: Jacobi or none
        a.precond = "jacobi"
    # the nonlinear workloads name no restart length: GMRES(30) stagnates on
    # the Richards L-scheme systems (67 restarts per solve at 96^3) and
    # GMRES(64) needs a fifth of the Arnoldi steps there (and 11 % fewer for
    # diffusion-reaction); the linear ones are GMRES(30)
    a.restart = a.restart or (30 if linear(a) else 64)
    return a


def linear(args):
    return args.workload in ("convdiff3d", "convdiff2d", "serve", "batch")


def inner_tol_for(args, s):
    if args.inner_tol is not None:
        return args.inner_tol
    if args.workload == "richards":
        return 1e-2       # L-scheme: linear outer convergence, loose inner solves suffice
    if not linear(args):
        return 1e-5 if args.precision == "fp64" else 1e-4     # Sec. 4.2: 1e-5
    if s > 1:
        return 1e-2                       # Sec. 4.1: loose inner solves for s > 1
    return 1e-10 if args.precision == "fp64" else 1e-5


def nl_stages(args):
    return 8          # diffreact: 4 SDIRK2 steps; richards: 8 implicit-Euler steps


# ----------------------------------------------------------------- oracle
def oracle_sample(args, n, reps=1):
    """Time the oracle on an n-cell-per-direction sample of the workload (this
    process runs with single-threaded BLAS). Returns time steps, cells, times."""
    import numpy as np
    import synth
    from oracle import coupling, fv, newton, slab
    s = args.s
    times = []
    if args.workload == "batch":
        # the first n slabs of the same seeded mix, solved one after another
        jobs = synth.batch_jobs(7, n)
        work = 0
        sample = []
        A, _, _ = coupling.implicit_euler()
        for j in jobs:
            w = synth.Workload("batch", j["dims"], "convdiff", j["s"], 1e-3, 1e-10, "jacobi",
                               batch_velocity(j["dims"]), "lognormal_iid", j["seed_coef"],
                               j["seed_rhs"])
            K = fv.convdiff_matrix(w.dims, synth.diffusion_field(w), w.velocity)
            A1, A2, _ = coupling.multistep_matrices(A, j["s"], w.tau)
            sample.append((K, w.n, A1, A2, synth.rhs_block(w)))
            work += w.n * j["s"]
        for _ in range(reps):
            t = time.perf_counter()
            for K, nn, A1, A2, B in sample:
                slab.slab_solve_global(K, np.ones(nn), A1, A2, B, None, tol=1e-10,
                                       precond="jacobi", restart=args.restart, ortho="mgs")
            times.append(time.perf_counter() - t)
        return {"n": work, "steps": 1, "times": times}
    if args.workload in ("convdiff3d", "convdiff2d", "serve"):
        if args.workload == "serve":
            s = 4                     # a mid-size request of the stream
        w = synth.convdiff_3d(n, s) if args.workload != "convdiff2d" else synth.convdiff_2d_64(s)
        if args.workload == "convdiff2d" and n != 64:
            w.dims = (n, n, 1)
        D = synth.diffusion_field(w)
        K = fv.convdiff_matrix(w.dims, D, w.velocity)
        A, _, _ = coupling.implicit_euler()
        A1, A2, _ = coupling.multistep_matrices(A, s, w.tau)
        B = synth.rhs_block(w)
        for _ in range(reps):
            t = time.perf_counter()
            if args.solver in ("global", "batch"):
                slab.slab_solve_global(K, np.ones(w.n), A1, A2, B, None, tol=w.tol,
                                       precond=args.precond, restart=args.restart)
            else:
                slab.slab_solve(K, np.ones(w.n), A1, A2, B, None, tol=w.tol,
                                inner_tol=1e-2 if s > 1 else 1e-10, precond=args.precond,
                                restart=args.restart, solver=args.solver)
            times.append(time.perf_counter() - t)
        return {"n": w.n, "steps": s, "times": times}
    if args.workload == "diffreact":
        dims = (n, n, 1)
        prob = newton.DiffReactProblem(dims)
        A, _, c = coupling.sdirk2()
        tau, y0, tol = 1e-2, np.full(n * n, 0.5), 1e-8
        G = nl_stages(args)
        for _ in range(reps):
            t = time.perf_counter()
            newton.pipelined_block_newton(prob, A, c, tau, y0, G, s, tol=tol, inner_tol=1e-5,
                                          precond=args.precond, restart=args.restart,
                                          solver=args.solver)
            times.append(time.perf_counter() - t)
        return {"n": n * n, "steps": G // 2, "times": times}
    dims = (n, n, n)
    w = synth.richards_3d(n, s)
    Ks = np.exp(2.0 * synth.correlated_field(w.seed_coef, dims[::-1], 8.0 * n / 96.0))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    prob = newton.RichardsProblem(dims, Ks, vg, 1.0 / 16.0)
    A, _, c = coupling.implicit_euler()
    z, _ = fv.richards_cells(dims)
    G = nl_stages(args)
    for _ in range(reps):
        t = time.perf_counter()
        newton.pipelined_block_newton(prob, A, c, 1.0 / 96.0, -z, G, s, tol=1e-5, inner_tol=1e-2,
                                      precond=args.precond, max_step=1.0, max_newton=150,
                                      lscheme_L=vg.lipschitz(), restart=args.restart,
                                      solver=args.solver)
        times.append(time.perf_counter() - t)
    return {"n": n ** 3, "steps": G, "times": times}


def oracle_sample_size(args):
    return {"convdiff3d": 48, "convdiff2d": 64, "diffreact": 160, "richards": 20,
            "serve": 32, "batch": 12}[args.workload]


def batch_velocity(dims):
    """Velocity of the batch mix: (1, 0.5) in 2-D, (1, 0.5, 0.25) in 3-D."""
    return (1.0, 0.5, 0.25) if dims[2] > 1 else (1.0, 0.5, 0.0)


def _oracle_cmd(args, n, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n), "--s", str(args.s),
           "--steps", str(reps), "--workload", args.workload, "--precond", args.precond,
           "--solver", args.solver, "--restart", str(args.restart)]
    return cmd, env


def run_oracle_subprocess(args, n, reps):
    cmd, env = _oracle_cmd(args, n, reps)
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_all_cores(args, n, cores=None):
    """The same oracle sample solved by one single-threaded process per host
    core, all at once: returns (cores, wall seconds, per-process results)."""
    cores = cores or os.cpu_count() or 1
    cmd, env = _oracle_cmd(args, n, 1)
    t = time.perf_counter()
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env) for _ in range(cores)]
    outs = []
    for pr in procs:
        o, e = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return cores, time.perf_counter() - t, outs


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
NOMINAL_HBM_GBS = 7900.0      # GB300 HBM3e, nominal (context for the measured peak)


def spbop_bytes(nnz, n, k, val_bytes=8, vec_bytes=8, idx_bytes=4, vector_reuse=True,
                write_result=True):
    """Bytes one sparse block operator product Z = A X with k columns moves
    (CSR): values and column indices once, the row pointer, X and Z. The
    defaults are the library's algorithmic count for its inner SpMM (X read
    once, Z written once). With vector_reuse=False every nonzero loads its k
    entries of X, and with no index bytes and no result writes this is the
    count of the paper's performance analysis (Sec. Performance analysis:
    one matrix entry and k block-vector entries per nonzero)."""
    b = nnz * (val_bytes + idx_bytes) + (n + 1) * idx_bytes
    b += (n if vector_reuse else nnz) * k * vec_bytes
    if write_result:
        b += n * k * vec_bytes
    return b


def spbop_ai(nnz, n, k, **kw):
    """Arithmetic intensity (flop per byte) of the sparse block product:
    2 k flops per nonzero over spbop_bytes."""
    return 2.0 * nnz * k / spbop_bytes(nnz, n, k, **kw)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def solver_label(args):
    return {"gmres": f"block GMRES({args.restart})", "cg": "block CG",
            "bicgstab": "block BiCGStab",
            "global": f"global GMRES({args.restart}) on the unsplit operator",
            "batch": f"global GMRES({args.restart}) on the unsplit operator in the batched "
                     f"persistent kernel"}[args.solver]


def solver_code(P, name):
    return {"gmres": P.PINT_SOLVER_GMRES, "cg": P.PINT_SOLVER_CG,
            "bicgstab": P.PINT_SOLVER_BICGSTAB, "global": P.PINT_SOLVER_GLOBAL,
            "batch": P.PINT_SOLVER_GLOBAL}[name]


# Files whose content fixes a kernel family's device code and launch shape:
# its translation unit, the shared internal header and the build (flags).
KERNEL_SOURCES = {
    "ilu": ("paper_2504_02117_gb300/csrc/ilu.cu", "paper_2504_02117_gb300/csrc/internal.h",
            "paper_2504_02117_gb300/build.py"),
    "spmm": ("paper_2504_02117_gb300/csrc/spmm.cu", "paper_2504_02117_gb300/csrc/internal.h",
             "paper_2504_02117_gb300/build.py"),
}


def source_hash(family):
    """Hash of the sources of one kernel family (KERNEL_SOURCES): a captured
    DRAM traffic figure is reported only while they are unchanged."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, rel), "rb") as fh:
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
    if not e or family not in KERNEL_SOURCES or e.get("source_hash") != source_hash(family):
        return None
    return e.get("dram_bytes_per_launch")


def roofline(fam, prof, hbm_peak, peak_kind, precision, workload, fp64_peak):
    tot_ms = prof["ms"]
    if tot_ms <= 0 or prof["launches"] == 0:
        return None
    per_launch_s = tot_ms / 1e3 / prof["launches"]
    bytes_pl = prof["bytes"] / prof["launches"]
    flops_pl = prof["flops"] / prof["launches"]
    gbs = bytes_pl / per_launch_s / 1e9
    t_mem = bytes_pl / (hbm_peak * 1e9)
    t_alu = flops_pl / (fp64_peak * 1e12) if precision == "fp64" else 0.0
    if t_alu > t_mem:
        ach = flops_pl / per_launch_s / 1e12
        return {"kernel": fam, "bound": "alu", "achieved": round(ach, 4),
                "peak": round(fp64_peak, 4), "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
                "peak_source": "measured float64 FMA rate (pint_fp64_fma_peak, this run)",
                "traffic": ncu_traffic(fam, workload),
                "algorithmic_bytes_per_launch": bytes_pl, "launches": prof["launches"],
                "avg_launch_us": per_launch_s * 1e6}
    return {"kernel": fam, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
            "frac_of_nominal": round(gbs / NOMINAL_HBM_GBS, 4),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "traffic": ncu_traffic(fam, workload), "algorithmic_bytes_per_launch": bytes_pl,
            "launches": prof["launches"], "avg_launch_us": per_launch_s * 1e6}


# ------------------------------------------------------------------ cases
class LinearCase:
    """One step = one slab solve of s coupled implicit-Euler steps."""

    def __init__(self, P, ctx, args):
        import numpy as np
        import torch
        import synth
        self.P, self.ctx, self.args = P, ctx, args
        s = args.s
        w = synth.convdiff_3d(args.n, s) if args.workload == "convdiff3d" else \
            synth.convdiff_2d_64(s)
        if args.workload == "convdiff2d":
            w.dims = (args.n, args.n, 1)
        self.w = w
        self.n, self.s, self.time_steps = w.n, s, s
        D = synth.diffusion_field(w).ravel()
        self.B = synth.rhs_block(w)
        self.op = P.pint_fv_convdiff(ctx, *w.dims, D, w.velocity)
        P.pint_set_coupling(ctx, self.op, (np.eye(s) - np.eye(s, k=-1)) / w.tau, np.eye(s))
        o = P.pint_opts_default()
        o.tol = w.tol
        o.inner_tol = inner_tol_for(args, s)
        o.precond = P.PINT_PC_ILU0 if args.precond == "ilu0" else P.PINT_PC_JACOBI
        o.precision = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}[args.precision]
        o.restart = args.restart
        o.solver = solver_code(P, args.solver)
        self.o = o
        self.Bd = torch.tensor(self.B, device="cuda", dtype=torch.float64)
        self.Y = torch.zeros(self.n, s, device="cuda", dtype=torch.float64)
        self.nnz = int(P.pint_operator_nnz(self.op))
        self.plan = None
        if args.solver == "batch":        # one slab, one cluster, a captured graph
            self.plan = P.BatchPlan(ctx, [(self.op, self.Bd, None, self.Y)], o,
                                    cluster_ctas=args.batch_cluster,
                                    cta_threads=args.batch_threads)

    def step(self):
        self.Y.zero_()
        if self.plan is not None:
            return self.plan.run()[0]
        return self.P.pint_solve_block(self.ctx, self.op, self.Bd, None, self.Y, self.o)

    def host_buffers(self):
        import torch
        self.Bh = torch.tensor(self.B, dtype=torch.float64).pin_memory()
        self.Yh = torch.empty(self.n, self.s, dtype=torch.float64).pin_memory()
        return self.Bh.numel() * 8, self.Yh.numel() * 8

    def e2e_step(self):
        self.Bd.copy_(self.Bh, non_blocking=True)
        st = self.step()
        self.Yh.copy_(self.Y, non_blocking=True)
        return st

    def describe(self):
        d = {"cells": self.n, "s": self.s, "nnz": self.nnz, "tau": self.w.tau,
             "tol": self.w.tol, "inner_tol": self.o.inner_tol, "restart": self.o.restart,
             "solver": self.args.solver}
        if self.plan is not None:
            d["launch_shape"] = self.plan.shape()
        return d

    def close(self):
        if self.plan is not None:
            self.plan.close()
        self.P.pint_operator_destroy(self.op)


class _AggStats:
    """pint_stats of a batch, summarised like one solve's (worst status and
    residual, summed steps and operations)."""

    def __init__(self, sts):
        self.sts = sts
        self.setup_ms = 0.0

    def as_dict(self, s=None):
        return {"status": max(x.status for x in self.sts),
                "outer_its": max(x.outer_its for x in self.sts),
                "inner_its": sum(x.inner_its for x in self.sts),
                "restarts": sum(x.restarts for x in self.sts),
                "col_relres": [max(max(x.col_relres) for x in self.sts)],
                "flops": sum(x.flops for x in self.sts), "solve_ms": self.sts[0].solve_ms,
                "max_inner_its": max(x.inner_its for x in self.sts)}


class BatchCase:
    """One step = one batched launch (a replay of the plan's captured graph)
    solving every slab of the seeded mix from Y = 0; the slabs' B and Y are
    views of two flat device buffers."""

    def __init__(self, P, ctx, args):
        import numpy as np
        import torch
        import synth
        self.P, self.ctx, self.args = P, ctx, args
        self.jobs = synth.batch_jobs(7, args.requests)
        counts = [j["dims"][0] * j["dims"][1] * j["dims"][2] * j["s"] for j in self.jobs]
        total = int(sum(counts))
        self.Bhost = np.empty(total)
        self.Bflat = torch.empty(total, device="cuda", dtype=torch.float64)
        self.Yflat = torch.zeros(total, device="cuda", dtype=torch.float64)
        self.ops, views, off = [], [], 0
        for j, cnt in zip(self.jobs, counts):
            w = synth.Workload("batch", j["dims"], "convdiff", j["s"], 1e-3, 1e-10, "jacobi",
                               batch_velocity(j["dims"]), "lognormal_iid", j["seed_coef"],
                               j["seed_rhs"])
            op = P.pint_fv_convdiff(ctx, *w.dims, synth.diffusion_field(w).ravel(), w.velocity)
            s = j["s"]
            P.pint_set_coupling(ctx, op, (np.eye(s) - np.eye(s, k=-1)) / w.tau, np.eye(s))
            self.Bhost[off:off + cnt] = synth.rhs_block(w).ravel()
            views.append((op, self.Bflat[off:off + cnt].view(w.n, s), None,
                          self.Yflat[off:off + cnt].view(w.n, s)))
            self.ops.append(op)
            off += cnt
        self.Bflat.copy_(torch.from_numpy(self.Bhost))
        o = P.pint_opts_default()
        o.tol = 1e-10
        o.precond = P.PINT_PC_JACOBI
        o.precision = P.PINT_FP64
        o.restart = args.restart
        self.o = o
        self.plan = P.BatchPlan(ctx, views, o, cluster_ctas=args.batch_cluster,
                                cta_threads=args.batch_threads)
        self.n, self.time_steps, self.s = total, 1, max(j["s"] for j in self.jobs)

    def step(self):
        self.Yflat.zero_()
        return _AggStats(self.plan.run())

    def host_buffers(self):
        import torch
        self.Bh = torch.from_numpy(self.Bhost).pin_memory()
        self.Yh = torch.empty(self.n, dtype=torch.float64).pin_memory()
        return self.Bh.numel() * 8, self.Yh.numel() * 8

    def e2e_step(self):
        self.Bflat.copy_(self.Bh, non_blocking=True)
        st = self.step()
        self.Yh.copy_(self.Yflat, non_blocking=True)
        return st

    def describe(self):
        import collections
        two = sum(1 for j in self.jobs if j["dims"][2] == 1)
        return {"slabs": len(self.jobs), "slabs_2d": two, "slabs_3d": len(self.jobs) - two,
                "dof_time_steps_per_launch": self.n,
                "s_counts": dict(sorted(collections.Counter(j["s"] for j in self.jobs).items())),
                "tol": 1e-10, "restart": self.o.restart, "solver": "batch",
                "launch_shape": self.plan.shape()}

    def close(self):
        self.plan.close()
        for op in self.ops:
            self.P.pint_operator_destroy(op)


class PipelineCase:
    """One step = Algorithm 1 over all stages of the run (pipelined windows)."""

    def __init__(self, P, ctx, args):
        import numpy as np
        import torch
        import synth
        self.P, self.ctx, self.args = P, ctx, args
        n, s = args.n, args.s
        self.s = s
        self.G = nl_stages(args)
        VG = (1.0, 2.0, 0.05, 0.4, 1.0 / 16.0)
        if args.workload == "diffreact":
            dims = (n, n, 1)
            self.prob = P.pint_problem_create(ctx, P.PINT_PROBLEM_DIFFREACT, *dims)
            self.A = np.array([[1 - 2 ** -0.5, 0.0], [2 ** -0.5, 1 - 2 ** -0.5]])
            self.c = np.array([1 - 2 ** -0.5, 1.0])
            self.tau, self.tol = 1e-2, 1e-8
            y0 = np.full(n * n, 0.5)
            self.time_steps = self.G // 2
            self.max_step = 0.0
            self.lscheme = 0.0
        else:
            dims = (n, n, n)
            w = synth.richards_3d(n, s)
            Ks = np.exp(2.0 * synth.correlated_field(w.seed_coef, dims[::-1], 8.0 * n / 96.0))
            self.Ksd = torch.tensor(Ks.ravel(), device="cuda", dtype=torch.float64)
            self.prob = P.pint_problem_create(ctx, P.PINT_PROBLEM_RICHARDS, *dims, params=VG,
                                              field=self.Ksd)
            self.A, self.c = np.array([[1.0]]), np.array([1.0])
            # Sec. 4.3: implicit Euler, tau = 1/96, the L-scheme with L the
            # Lipschitz constant of theta, outer tolerance 1e-5
            self.tau, self.tol = 1.0 / 96.0, 1e-5
            z = (np.arange(n) + 0.5) / n
            y0 = -np.broadcast_to(z[:, None, None], (n, n, n)).ravel().copy()
            self.time_steps = self.G
            self.max_step = 1.0
            self.lscheme = 0.0 if args.linearisation == "newton" else -1.0
        self.n = int(np.prod(dims))
        self.y0 = y0
        self.y0d = torch.tensor(y0, device="cuda", dtype=torch.float64)
        self.out = torch.zeros(self.n, self.G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = self.tol
        o.inner_tol = inner_tol_for(args, s)
        o.max_outer = 150 if self.lscheme else 60
        o.max_step = self.max_step
        o.lscheme_L = self.lscheme
        o.precond = P.PINT_PC_ILU0 if args.precond == "ilu0" else P.PINT_PC_JACOBI
        o.precision = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}[args.precision]
        o.restart = args.restart
        o.solver = solver_code(P, args.solver)
        self.o = o
        self.nnz = int(P.pint_operator_nnz(P.pint_problem_operator(self.prob)))

    def step(self):
        return self.P.pint_pipeline_run(self.ctx, self.prob, self.A, self.c, self.tau, self.s,
                                        self.y0d, self.G, self.out, self.o)

    def host_buffers(self):
        import torch
        self.y0h = torch.tensor(self.y0, dtype=torch.float64).pin_memory()
        self.outh = torch.empty(self.n, self.G, dtype=torch.float64).pin_memory()
        return self.y0h.numel() * 8, self.outh.numel() * 8

    def e2e_step(self):
        self.y0d.copy_(self.y0h, non_blocking=True)
        st = self.step()
        self.outh.copy_(self.out, non_blocking=True)
        return st

    def describe(self):
        return {"cells": self.n, "s": self.s, "stages": self.G, "nnz": self.nnz, "tau": self.tau,
                "tol": self.tol, "inner_tol": self.o.inner_tol, "restart": self.o.restart,
                "max_step": self.max_step,
                "linearisation": "L-scheme (L = Lipschitz constant of theta)" if self.lscheme
                else "simplified Newton", "solver": self.args.solver}

    def close(self):
        self.P.pint_problem_destroy(self.prob)


# ------------------------------------------------------------------ main
def max_over_ranks(ms, dist=None, device="cuda"):
    """The slowest rank's time (every rank gets it); `ms` itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, time_steps, cells, ms):
    """Whole-job time-step*DOF/s of `world` independent replicas, each
    solving `steps` slabs of `time_steps` steps on `cells` cells in `ms`."""
    return world * steps * time_steps * cells / (ms / 1e3)


def main():
    args = parse()
    if args.oracle_sample:
        r = oracle_sample(args, args.oracle_sample, max(1, args.steps))
        print(json.dumps(r))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    desc = WORKLOADS[args.workload][4].format(n=args.n, pc=args.precond,
                                             solver=solver_label(args), requests=args.requests,
                                             lin="Newton" if args.linearisation == "newton"
                                             else "L-scheme")
    wl_name = f"{args.workload}_n{args.n}_s{args.s}_{args.precond}"
    if args.workload == "richards" and args.linearisation == "newton":
        wl_name += "_newton"
    if args.workload == "batch":
        wl_name = f"batch_{args.requests}slabs_jacobi"
    elif args.solver == "batch":
        wl_name += "_batchkernel"

    if args.impl == "reference":
        if rank != 0:
            return
        return reference_arm(args, wl_name, desc, world)

    # CPU baseline first: a spawned single-threaded process, before any GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        samp = oracle_sample_size(args)
        try:
            r = run_oracle_subprocess(args, samp, 1)
            v1 = r["steps"] * r["n"] / min(r["times"])
            cores, wall, outs = run_oracle_all_cores(args, samp)
            work = sum(o["steps"] * o["n"] for o in outs)
            cpu = {"value": work / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{cores} single-threaded oracle processes (FP64, {args.precond}, "
                             f"same recipe), one per host core, each solving the same "
                             f"{r['n']}-cell sample of {r['steps']} time steps at once: "
                             f"{wall:.1f} s wall",
                   "one_core": {"value": v1, "cores": 1,
                                "sample": f"one oracle run on {r['n']} cells, {r['steps']} "
                                          f"time steps: {min(r['times']):.1f} s"}}
        except Exception as e:          # report, do not hide
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"failed: {e}"[:300]}

    if args.workload == "serve":
        return serve_main(args, world, rank, local, cpu, desc)

    import torch
    import paper_2504_02117_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = P.pint_create(local)
    fp64_peak = P.pint_fp64_fma_peak(ctx)
    if args.workload == "batch":
        case = BatchCase(P, ctx, args)
    elif linear(args):
        case = LinearCase(P, ctx, args)
    else:
        case = PipelineCase(P, ctx, args)
    stream = torch.cuda.current_stream()

    # set-up (ILU factorisation happens on the first solve): untimed
    t0 = time.perf_counter()
    st0 = case.step()
    setup_s = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        case.step()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------------------------------------------------- timed region
    # K steps with the profiler off give `value`; K more steps with the
    # library's per-family CUDA-event profiler on give the roofline table
    l0 = P.pint_kernel_launches(ctx)
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            stats.append(case.step().as_dict(case.s))
        ev1.record(stream)
        barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    launches = P.pint_kernel_launches(ctx) - l0
    value = replica_throughput(world, args.steps, case.time_steps, case.n, elapsed_ms)
    converged = all(st["status"] == 0 for st in stats)

    P.pint_profile_reset(ctx)
    P.pint_profile_enable(ctx, True)
    barrier()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        case.step()
    p1.record(stream)
    barrier()
    profiled_ms = p0.elapsed_time(p1) / args.steps
    P.pint_profile_enable(ctx, False)
    fams = {name: P.pint_profile_read(ctx, k) for k, name in enumerate(P.KERNEL_FAMILIES)}

    # ------------------------------------------------------------- e2e leg
    e2e = None
    if not args.no_e2e:
        bi, bo = case.host_buffers()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            case.e2e_step()
        e1.record(stream)
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        e2e = {"value": replica_throughput(world, args.steps, case.time_steps, case.n, e_ms),
               "unit": UNIT, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
               "ms_per_step": e_ms / args.steps}

    if rank != 0:
        case.close()
        P.pint_destroy(ctx)
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---------------------------------------- the same workload in pure FP64
    fp64 = bf16 = glob = None
    if args.precision != "fp64" and not args.no_fp64:
        fp64 = precision_variant(P, case, args, stream, "fp64")
        if args.precision == "fp32":
            bf16 = precision_variant(P, case, args, stream, "bf16")
    batchv = None
    if linear(args) and args.solver == "gmres" and not args.no_fp64:
        glob = solver_variant(P, case, args, stream, "global")
        if args.workload == "convdiff2d":
            batchv = batch_variant(P, ctx, case, args, stream, fp64_peak)

    hbm_peak, peak_kind = measured_peaks()
    total_prof = sum(f["ms"] for f in fams.values()) or 1.0
    dominant = max((k for k in fams if k not in ("vec",)), key=lambda k: fams[k]["ms"])
    kernels = {}
    for k, f in fams.items():
        if f["launches"]:
            kernels[k] = {"launches": f["launches"], "ms": round(f["ms"], 3),
                          "share": round(f["ms"] / total_prof, 4),
                          "GB/s": round(f["bytes"] / max(f["ms"], 1e-9) / 1e6, 1)}
    cfg = {"workload": wl_name, "description": desc, "precision": args.precision,
           "precond": args.precond, "time_steps_per_step": case.time_steps,
           "parallelism": f"replicas x{world}",
           "l2": "inputs larger than L2 (matrix + Krylov basis >> 129 MB), no flush"
           if case.n >= 1 << 20 else "small workload: partly L2-resident, no flush"}
    cfg.update(case.describe())
    if args.solver == "batch":
        rl = batch_roofline(stats, elapsed_ms / args.steps, fp64_peak)
        kernels = {"k_slab_queue": {"launches": args.steps, "ms": round(elapsed_ms, 3),
                                    "share": 1.0, "note": "one graph replay per step; the "
                                    "step time also holds the Y reset and the status read"}}
        spmm_rl = None
    else:
        rl = roofline(dominant, fams[dominant], hbm_peak, peak_kind, args.precision, wl_name,
                      fp64_peak)
        spmm_rl = roofline("spmm", fams["spmm"], hbm_peak, peak_kind, args.precision, wl_name,
                           fp64_peak)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else f"f64+{args.precision}",
        "data": "synthetic", "config": cfg,
        "roofline": rl,
        "spmm_roofline": spmm_rl,
        "fp64_peak": {"tflops": round(fp64_peak, 4), "source": "pint_fp64_fma_peak (measured "
                      "on this GPU in this run)", "nominal_tflops": FP64_NOMINAL_TFLOPS},
        "kernels": kernels, "profiled_ms_per_step": profiled_ms,
        "iterations": {"outer": stats[-1]["outer_its"], "inner": stats[-1]["inner_its"],
                       "restarts": stats[-1]["restarts"]},
        "converged": converged, "max_col_relres": max(max(st["col_relres"]) for st in stats),
        "setup": {"first_step_s": setup_s, "precond_setup_ms": st0.setup_ms},
        "fp64": fp64, "bf16": bf16, "global_fp64": glob, "batch_kernel_fp64": batchv,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk.summary(), "impl": "pint",
    }
    if linear(args) and args.solver != "batch":
        out["spmm_full_width"] = spmm_full_width(P, ctx, case, args.precision, hbm_peak)
    if not args.no_sweep and args.workload == "convdiff3d" and args.solver != "global":
        out["sweep"] = sweep(P, ctx, args, case.w, fp64_peak)
        out["sweep_summary"] = sweep_summary(out["sweep"])
    if not args.no_other and args.workload == "convdiff3d":
        out["other_configs"] = other_configs(P, ctx, fp64_peak, max(2, min(args.steps, 5)))
    print(json.dumps(out), flush=True)
    case.close()
    P.pint_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def other_configs(P, ctx, fp64_peak, steps):
    """Compact legs of the other configurations, measured in the same run as
    the headline (each: set-up and one warm-up untimed, then `steps` timed
    steps with CUDA events): the headline slab with block BiCGStab inner
    solves (the paper's solver for this problem), the 64 x 64 slab through
    the batched kernel (one cluster), 512 uneven slabs in one batched launch,
    and the 512^2 diffusion-reaction run of Algorithm 1."""
    import torch
    legs = {
        "convdiff3d_128_s8_bicgstab_fp32": ["--workload", "convdiff3d", "--solver", "bicgstab"],
        "convdiff2d_64_s4_batch_kernel": ["--workload", "convdiff2d", "--solver", "batch"],
        "batch_512_slabs": ["--workload", "batch", "--requests", "512"],
        "diffreact_512_fp32": ["--workload", "diffreact"],
    }
    out = {}
    stream = torch.cuda.current_stream()
    for name, argv in legs.items():
        case = None
        try:
            a = parse(argv + ["--steps", str(steps)])
            if a.workload == "batch":
                case = BatchCase(P, ctx, a)
            elif linear(a):
                case = LinearCase(P, ctx, a)
            else:
                case = PipelineCase(P, ctx, a)
            case.step()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sts = [case.step().as_dict(case.s) for _ in range(steps)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            d = {"value": case.time_steps * case.n / (ms / 1e3), "unit": UNIT,
                 "ms_per_step": ms, "steps": steps, "precision": a.precision,
                 "solver": solver_label(a), "precond": a.precond,
                 "converged": all(x["status"] == 0 for x in sts),
                 "max_col_relres": max(max(x["col_relres"]) for x in sts),
                 "inner": sts[-1]["inner_its"]}
            if a.solver == "batch":
                d["roofline"] = batch_roofline(sts, ms, fp64_peak)
                d["launch_shape"] = case.plan.shape()
            out[name] = d
        except Exception as e:          # report, do not hide
            out[name] = {"value": None, "error": str(e)[:300]}
        finally:
            if case is not None:
                case.close()
    return out


def batch_roofline(stats, ms_per_step, fp64_peak):
    """The batched kernel is bound by the float64 pipe (about 1/64 of the
    float32 rate on this GPU), not by HBM: achieved = the algorithmic float64
    operations the kernel counted (FMA = 2; plain adds, multiplies and square
    roots 1 each, although each takes a full FMA issue slot) per step over the
    step time, against the measured float64 FMA rate."""
    fl = stats[-1].get("flops") or 0.0
    if fl <= 0 or ms_per_step <= 0:
        return None
    ach = fl / (ms_per_step / 1e3) / 1e12
    return {"kernel": "k_slab_queue", "bound": "alu", "achieved": round(ach, 4),
            "peak": round(fp64_peak, 4), "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4),
            "peak_source": "measured float64 FMA rate (pint_fp64_fma_peak, this run)",
            "flops_per_step": fl, "traffic": None, "launches": 1,
            "avg_launch_us": ms_per_step * 1e3,
            "note": "step time (graph replay + Y reset + status read) as the launch time"}


def batch_variant(P, ctx, case, args, stream, fp64_peak):
    """The same slab through the batched persistent kernel (one cluster, a
    captured graph), float64 + Jacobi: one warm-up, then as many timed steps
    as the headline."""
    import torch
    plan = None
    try:
        o = P.pint_opts_default()
        o.tol = case.o.tol
        o.precond = P.PINT_PC_JACOBI
        o.precision = P.PINT_FP64
        o.restart = case.o.restart
        plan = P.BatchPlan(ctx, [(case.op, case.Bd, None, case.Y)], o)
        case.Y.zero_()
        plan.run()
        k = max(1, args.steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sts = []
        for _ in range(k):
            case.Y.zero_()
            sts.append(plan.run()[0].as_dict(case.s))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        return {"value": case.time_steps * case.n / (ms / 1e3), "unit": UNIT,
                "ms_per_step": ms, "steps": k, "launch_shape": plan.shape(),
                "solver": f"global GMRES({o.restart}) + Jacobi in the batched persistent kernel",
                "outer": sts[-1]["outer_its"], "inner": sts[-1]["inner_its"],
                "converged": all(x["status"] == 0 for x in sts),
                "max_col_relres": max(max(x["col_relres"]) for x in sts),
                "roofline": batch_roofline(sts, ms, fp64_peak)}
    except Exception as e:              # report, do not hide
        return {"value": None, "error": str(e)[:300]}
    finally:
        if plan is not None:
            plan.close()


def solver_variant(P, case, args, stream, solver):
    """Time the same slab with another solver (one warm-up, then as many timed
    steps as the headline): "global" is global GMRES on the unsplit operator,
    float64."""
    import torch
    saved = (case.o.solver, case.o.precision)
    case.o.solver = solver_code(P, solver)
    if solver == "global":
        case.o.precision = P.PINT_FP64
    try:
        case.step()
        k = max(1, args.steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sts = [case.step().as_dict(case.s) for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        return {"value": case.time_steps * case.n / (ms / 1e3), "unit": UNIT,
                "ms_per_step": ms, "steps": k, "solver": solver_label(
                    argparse.Namespace(**dict(vars(args), solver=solver))),
                "outer": sts[-1]["outer_its"], "inner": sts[-1]["inner_its"],
                "converged": all(x["status"] == 0 for x in sts),
                "max_col_relres": max(max(x["col_relres"]) for x in sts)}
    except Exception as e:              # report, do not hide
        return {"value": None, "error": str(e)[:300]}
    finally:
        case.o.solver, case.o.precision = saved


def spmm_full_width(P, ctx, case, prec, hbm_peak, reps=20):
    """The inner SpMM (Z = J X) alone at the workload's full block width, in
    the inner-solve precision: `reps` launches alternating between two input /
    output pairs (together far larger than L2), timed by the library's
    CUDA-event profiler on the launching stream; bytes are the kernel's own
    algorithmic bytes (the library's count). The in-solve figure
    (`spmm_roofline`) averages over narrowed widths as well."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}[prec]
    g = torch.Generator(device="cuda").manual_seed(7)
    bufs = [(torch.rand(case.n, case.s, device="cuda", dtype=dt, generator=g),
             torch.empty(case.n, case.s, device="cuda", dtype=dt)) for _ in range(2)]

    def apply(i):
        X, Z = bufs[i % 2]
        if prec == "fp64":
            P.pint_inner_apply(ctx, case.op, X, Z)
        else:
            P.pint_inner_apply_lowp(ctx, case.op, code, X, Z)
    for i in range(3):
        apply(i)
    torch.cuda.synchronize()
    P.pint_profile_reset(ctx)
    P.pint_profile_enable(ctx, True)
    for i in range(reps):
        apply(i)
    P.pint_profile_enable(ctx, False)
    r = P.pint_profile_read(ctx, 1)
    per_s = r["ms"] / 1e3 / r["launches"]
    b = r["bytes"] / r["launches"]
    gbs = b / per_s / 1e9
    vb = {"fp64": 8, "fp32": 4, "bf16": 2}[prec]
    xb = 8 if prec == "fp64" else 4
    # the format the kernel reads: 8 stencil coefficients per row for grid
    # operators (SELL-32 values and indices otherwise), X read, Z written once
    fmt = 8 * vb * case.n + 2 * xb * case.n * case.s
    return {"s": case.s, "precision": prec, "bound": "hbm", "achieved": round(gbs, 1),
            "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
            "algorithmic_bytes_per_launch": b, "avg_launch_us": per_s * 1e6,
            "launches": r["launches"],
            "format_bytes_per_launch": fmt,
            "format_GBs": round(fmt / per_s / 1e9, 1),
            "format_frac": round(fmt / per_s / 1e9 / hbm_peak, 4),
            "note": "achieved: CSR-form algorithmic bytes of the product (values + int32 "
                    "indices, row pointer, X read and Z written once) per launch time; "
                    "format_*: the stencil form's own bytes (8 coefficients per row)"}


def precision_variant(P, case, args, stream, prec="fp64"):
    """Time the same step with another inner-solve precision (one warm-up,
    then as many timed steps as the headline): FP64 is the "mixed vs FP64"
    half of the metric, BF16 the bfloat16-matrix variant of the mixed path."""
    import torch
    prec0, tol0 = case.o.precision, case.o.inner_tol
    case.o.precision = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}[prec]
    ns = argparse.Namespace(**vars(args))
    ns.precision = prec
    case.o.inner_tol = inner_tol_for(ns, case.s)
    try:
        case.step()
        k = max(1, args.steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sts = [case.step().as_dict(case.s) for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        return {"value": case.time_steps * case.n / (ms / 1e3), "unit": UNIT,
                "ms_per_step": ms, "steps": k, "inner_tol": case.o.inner_tol,
                "outer": sts[-1]["outer_its"], "inner": sts[-1]["inner_its"],
                "converged": all(x["status"] == 0 for x in sts),
                "max_col_relres": max(max(x["col_relres"]) for x in sts)}
    except Exception as e:              # report, do not hide
        return {"value": None, "error": str(e)[:300]}
    finally:
        case.o.precision, case.o.inner_tol = prec0, tol0


def sweep(P, ctx, args, w0, fp64_peak):
    """One timed solve per (precision, s) on the same grid (after one warm-up
    solve each): time-step*DOF/s, SpMM GB/s and the SpMM's s-dependent
    arithmetic-intensity roofline (flop per byte, achieved and attainable
    GFLOP/s against the measured HBM peak, and the FP64 rate in FP64)."""
    import numpy as np
    import torch
    import synth
    res = []
    hbm_peak, _ = measured_peaks()
    D = synth.diffusion_field(w0).ravel()
    for prec_name in ("fp64", "fp32"):
        for s in (1, 2, 4, 8, 16):
            w = synth.convdiff_3d(args.n, s)
            w.dims = w0.dims
            op = P.pint_fv_convdiff(ctx, *w.dims, D, w.velocity)
            P.pint_set_coupling(ctx, op, (np.eye(s) - np.eye(s, k=-1)) / w.tau, np.eye(s))
            o = P.pint_opts_default()
            o.tol = w.tol
            ns = argparse.Namespace(**vars(args))
            ns.precision = prec_name
            o.inner_tol = inner_tol_for(ns, s)
            o.precond = P.PINT_PC_ILU0
            o.precision = P.PINT_FP64 if prec_name == "fp64" else P.PINT_FP32
            o.restart = args.restart
            o.solver = solver_code(P, args.solver)
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
            gbs = sp["bytes"] / max(sp["ms"], 1e-9) / 1e6
            eb = 8 if prec_name == "fp64" else 4
            nnz = int(P.pint_operator_nnz(op))
            # over all SpMM launches of the solve (narrowed inner solves launch
            # narrower, lower-intensity products) and for a full-width launch
            ai = sp["flops"] / max(sp["bytes"], 1.0)
            ai_full = spbop_ai(nnz, w.n, s, val_bytes=eb, vec_bytes=eb)
            roof = hbm_peak * ai
            res.append({"precision": prec_name, "s": s, "value": s * w.n / dt,
                        "solve_s": dt, "outer": st.outer_its, "inner": st.inner_its,
                        "status": st.status, "spmm_GBs": gbs,
                        "spmm_ai_flop_per_byte": ai, "spmm_ai_full_width": ai_full,
                        "spmm_gflops": sp["flops"] / max(sp["ms"], 1e-9) / 1e6,
                        "spmm_roof_gflops": min(roof, 1e3 * fp64_peak)
                        if prec_name == "fp64" else roof})
            P.pint_operator_destroy(op)
            del Bd, Y
    return res


def sweep_summary(rows):
    """Per precision: time-step*DOF/s at s = 8 over s = 1 (the s-scaling
    target is >= 3) and the best width."""
    out = {}
    for prec in sorted({r["precision"] for r in rows}):
        v = {r["s"]: r["value"] for r in rows if r["precision"] == prec and r["status"] == 0}
        if 1 in v and 8 in v:
            best = max(v, key=v.get)
            out[prec] = {"s8_over_s1": round(v[8] / v[1], 3), "best_s": best,
                         "best_over_s1": round(v[best] / v[1], 3)}
    return out


def serve_main(args, world, rank, local, cpu, desc):
    """The serving workload: one seeded Poisson stream of slab-solve requests
    per GPU through the continuous-batching loop; value = time steps x cells
    of all completed requests / makespan. Every request's latency includes
    the upload of its inputs and the download of its solution (e2e)."""
    import torch
    import synth
    import paper_2504_02117_gb300 as P
    from paper_2504_02117_gb300 import serve

    torch.cuda.set_device(local)
    cache = {}

    def make(spec):
        key = (spec["n"], spec["s"])
        if key not in cache:            # the clients' data, seeded per shape
            w = synth.convdiff_3d(spec["n"], spec["s"])
            cache[key] = (w, synth.diffusion_field(w), synth.rhs_block(w))
        w, D, B = cache[key]
        ns = argparse.Namespace(**vars(args))
        ns.precision = spec["precision"]
        return serve.SlabRequest(rid=spec["rid"], arrival=spec["arrival"], dims=w.dims,
                                 s=spec["s"], precision=spec["precision"], D=D, B=B,
                                 velocity=w.velocity, tau=w.tau, tol=w.tol,
                                 inner_tol=inner_tol_for(ns, spec["s"]), restart=args.restart,
                                 solver=args.solver)

    grids = tuple(g for g in (32, 48, 64, 96, 128) if g <= args.n)
    specs = synth.request_stream(5 + rank, args.requests, args.rate, grids=grids)
    reqs = [make(sp) for sp in specs]
    srv = serve.SlabServer(slots=args.slots, device=local, keep_results=True,
                           batch_lane=not args.no_batch_lane,
                           batch_max_unknowns=args.batch_max_unknowns)
    try:
        warm = [make({"rid": -1 - i, "arrival": 0.0, "n": grids[0], "s": w, "precision": p})
                for i, (w, p) in enumerate([(2, "fp32"), (4, "fp64"), (8, "fp32"), (16, "fp64")])]
        srv.run(warm[:max(1, args.warmup)])
        with ClockSampler(torch.cuda.current_device()) as clk:
            summ = srv.run(reqs)
        launches = sum(int(P.pint_kernel_launches(c)) for c in srv._ctx if c is not None)
        if srv._bctx is not None:
            launches += int(P.pint_kernel_launches(srv._bctx))
    finally:
        srv.close()
    dist = None
    if world > 1:                       # replicas: one stream per GPU, slowest rank's span
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    span = max_over_ranks(summ["makespan_s"], dist, "cuda")
    if dist is not None:
        dist.destroy_process_group()
    done = [r for r in reqs if r.status == 0]
    work = sum(r.s * r.cells for r in done)
    value = world * work / span if span > 0 else None
    if rank != 0:
        return
    h2d = sum(r.B.nbytes + r.D.nbytes for r in done)
    d2h = sum(r.Y.nbytes for r in done if r.Y is not None)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": args.warmup, "ms_per_step": span * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+fp32/f64", "data": "synthetic",
        "config": {"workload": f"serve_{args.requests}req_rate{args.rate:g}_slots{args.slots}"
                               + ("" if args.no_batch_lane else "_batchlane"),
                   "batch_lane": None if args.no_batch_lane else
                   {"max_unknowns": args.batch_max_unknowns, "precision": "fp64",
                    "method": "global GMRES + Jacobi, one launch per batch, 8-CTA clusters"},
                   "description": desc, "grids": list(grids),
                   "widths": [2, 4, 8, 16], "precisions": ["fp32", "fp64"],
                   "restart": args.restart, "parallelism": f"replicas x{world}",
                   "l2": "mixed request sizes, no flush"},
        "latency": {"p50_ms": 1e3 * summ["p50_latency_s"], "p99_ms": 1e3 * summ["p99_latency_s"],
                    "p50_queue_ms": 1e3 * summ["p50_queue_s"],
                    "p99_queue_ms": 1e3 * summ["p99_queue_s"]},
        "serving": summ, "roofline": None,
        "roofline_note": "per-kernel rooflines: the convdiff3d workload",
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches, "clocks": clk.summary(), "impl": "pint",
    }
    print(json.dumps(out), flush=True)


def reference_arm(args, wl_name, desc, world):
    """The oracle as it stands, timed on this host's cores, on a bounded
    sample of the workload per step (the same sample as cpu_baseline)."""
    samp = oracle_sample_size(args)
    r = run_oracle_subprocess(args, samp, args.warmup + args.steps)
    times = r["times"][args.warmup:]
    per = statistics.mean(times)
    v = r["steps"] * r["n"] / per
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl_name, "description": desc, "sample_cells": r["n"],
                      "s": args.s},
           "impl": "reference",
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"oracle run on {r['n']} cells ({r['steps']} time steps) "
                                      f"per step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
