"""Measured choice of the block width, inner solver and inner precision for
time-slab solves.

How many time steps s to couple into one block solve (the block width), the
inner block solver and the inner precision all decide the throughput of the
vectorised method, and the best choice differs between problems and
precisions: on a 128^3 convection-diffusion slab with ILU(0), FP32 block
GMRES peaks at s = 8 and FP64 block BiCGStab at s = 4. The autotuner times
one slab solve per candidate (after a warm-up solve that builds the
operator's preconditioner and work space) and keeps the fastest in
time-step*DOF/s among the candidates that converge; a candidate whose first
measurement falls below `prune` times the best first measurement is not
measured again. Choices are kept in a JSON cache keyed by the problem's shape
and the device.

The measurement is a callable candidate -> dict(value, converged, ...), so
the search itself runs without a GPU; `slab_measure` builds the GPU one.

The same search picks the launch shape of the batched persistent solver
(`BatchShape`: CTAs per cluster and threads per CTA) for a given set of jobs:
`batch_measure` times one run of a resident plan per shape. The library's own
rule (pint_batch_auto_cluster / _threads) is fitted to such sweeps; the
autotuner measures the job set at hand instead.
"""
from __future__ import annotations

import dataclasses
import json
import os
import statistics
from typing import Callable, Iterable, Optional

SOLVERS = ("gmres", "bicgstab", "cg")
PRECISIONS = ("fp32", "bf16", "fp64")


@dataclasses.dataclass(frozen=True)
class Candidate:
    s: int                        # coupled time steps (block width)
    solver: str = "gmres"         # inner block solver: "gmres", "bicgstab" or "cg"
    precision: str = "fp32"       # inner precision: "fp32", "bf16" or "fp64"
    restart: int = 30             # GMRES restart length (BiCGStab needs >= 8)

    def __post_init__(self):
        if self.s < 1 or self.solver not in SOLVERS or self.precision not in PRECISIONS:
            raise ValueError(f"invalid candidate {self}")

    def key(self) -> str:
        return f"s{self.s}_{self.solver}_{self.precision}_m{self.restart}"


@dataclasses.dataclass(frozen=True)
class BatchShape:
    cluster_ctas: int             # CTAs per cluster (one job per cluster at a time)
    cta_threads: int = 512        # threads per CTA

    def __post_init__(self):
        if not 1 <= self.cluster_ctas <= 16 or self.cta_threads not in (128, 256, 512):
            raise ValueError(f"invalid batch shape {self}")

    def key(self) -> str:
        return f"c{self.cluster_ctas}_t{self.cta_threads}"


def batch_shapes(clusters: Iterable[int] = (1, 2, 4, 8, 16),
                 threads: Iterable[int] = (512, 256)) -> list:
    """All combinations, clusters innermost."""
    return [BatchShape(c, t) for t in threads for c in clusters]


def grid(widths: Iterable[int] = (1, 2, 4, 8, 16), solvers: Iterable[str] = ("gmres", "bicgstab"),
         precisions: Iterable[str] = ("fp32",), restart: int = 30) -> list:
    """All combinations, widths innermost."""
    return [Candidate(s, so, p, restart) for so in solvers for p in precisions for s in widths]


def autotune(measure: Callable[[Candidate], dict], candidates: Iterable[Candidate],
             repeats: int = 3, prune: float = 0.5):
    """Measure every candidate once, repeat the ones within `prune` of the
    best first measurement up to `repeats` times, rank by the median.
    Returns (best candidate or None, ranked table of dicts with keys
    candidate, values, value, converged, pruned, last)."""
    table = []
    best_first = 0.0
    for c in candidates:
        r = measure(c)
        ok = bool(r.get("converged", False))
        e = {"candidate": c, "values": [float(r["value"])] if ok else [], "converged": ok,
             "pruned": False, "last": r}
        if ok:
            best_first = max(best_first, e["values"][0])
        table.append(e)
    for e in table:
        if not e["converged"]:
            continue
        if e["values"][0] < prune * best_first:
            e["pruned"] = True
            continue
        for _ in range(repeats - 1):
            r = measure(e["candidate"])
            e["last"] = r
            if not r.get("converged", False):
                e["converged"] = False
                break
            e["values"].append(float(r["value"]))
    for e in table:
        e["value"] = statistics.median(e["values"]) if e["converged"] else 0.0
    ranked = sorted(table, key=lambda e: -e["value"])
    best = ranked[0]["candidate"] if ranked and ranked[0]["value"] > 0.0 else None
    return best, ranked


class TuneCache:
    """Chosen candidates by problem key, in a JSON file (written atomically)."""

    def __init__(self, path: str):
        self.path = path
        self.data = {}
        if os.path.exists(path):
            with open(path) as fh:
                self.data = json.load(fh)

    @staticmethod
    def key(dims, nnz: int, precond: str, tol: float, device: str) -> str:
        return f"{'x'.join(str(int(d)) for d in dims)}_nnz{int(nnz)}_{precond}_tol{tol:g}_{device}"

    def get(self, key: str) -> Optional[Candidate]:
        e = self.data.get(key)
        return Candidate(**e["candidate"]) if e and "candidate" in e else None

    def put(self, key: str, cand: Candidate, value: float):
        self.data[key] = {"candidate": dataclasses.asdict(cand), "value": float(value)}
        self._write()

    @staticmethod
    def batch_key(sizes, device: str) -> str:
        """A batch by its jobs' N s values (count, total, largest)."""
        sizes = [int(x) for x in sizes]
        return f"batch_{len(sizes)}jobs_sum{sum(sizes)}_max{max(sizes)}_{device}"

    def get_batch(self, key: str) -> Optional[BatchShape]:
        e = self.data.get(key)
        return BatchShape(**e["shape"]) if e and "shape" in e else None

    def put_batch(self, key: str, shape: BatchShape, value: float):
        self.data[key] = {"shape": dataclasses.asdict(shape), "value": float(value)}
        self._write()

    def _write(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(self.data, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def inner_tol(s: int, precision: str) -> float:
    """Inner tolerance of a linear slab: 1e-2 for coupled steps (Sec. 4.1);
    a single step is solved by the inner solve itself (1e-10 in FP64, 1e-5
    with a low-precision inner solve and FP64 refinement)."""
    if s > 1:
        return 1e-2
    return 1e-10 if precision == "fp64" else 1e-5


def slab_measure(ctx, dims, D, velocity, tau: float, rhs: Callable[[int], object],
                 tol: float = 1e-10, precond: str = "ilu0", device: int = 0):
    """The GPU measurement: a slab of c.s implicit-Euler steps of the
    finite-volume convection-diffusion operator on `dims` (cell field D,
    velocity), right-hand side rhs(s) (N x s float64 host array), Y0 = 0;
    one warm-up solve, then one solve timed with CUDA events on the current
    stream. value = s * N / seconds (time-step*DOF/s)."""
    import numpy as np
    import torch

    import paper_2504_02117_gb300 as P

    n = int(np.prod(dims))
    pc = {"ilu0": P.PINT_PC_ILU0, "jacobi": P.PINT_PC_JACOBI, "none": P.PINT_PC_NONE}[precond]
    prec = {"fp64": P.PINT_FP64, "fp32": P.PINT_FP32, "bf16": P.PINT_BF16}
    solver = {"gmres": P.PINT_SOLVER_GMRES, "bicgstab": P.PINT_SOLVER_BICGSTAB,
              "cg": P.PINT_SOLVER_CG}
    dev = f"cuda:{device}"
    D = np.ascontiguousarray(D, dtype=np.float64).ravel()

    def measure(c: Candidate) -> dict:
        op = P.pint_fv_convdiff(ctx, *dims, D, velocity)
        try:
            A1 = (np.eye(c.s) - np.eye(c.s, k=-1)) / tau
            P.pint_set_coupling(ctx, op, A1, np.eye(c.s))
            B = torch.as_tensor(np.ascontiguousarray(rhs(c.s)), dtype=torch.float64).to(dev)
            Y = torch.zeros(n, c.s, device=dev, dtype=torch.float64)
            o = P.pint_opts_default()
            o.tol = tol
            o.inner_tol = inner_tol(c.s, c.precision)
            o.precond = pc
            o.precision = prec[c.precision]
            o.solver = solver[c.solver]
            o.restart = c.restart
            try:
                P.pint_solve_block(ctx, op, B, None, Y, o)
                Y.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                st = P.pint_solve_block(ctx, op, B, None, Y, o)
                e1.record()
                torch.cuda.synchronize()
            except P.PintError as err:
                return {"value": 0.0, "converged": False, "status": err.code, "error": str(err)}
            ms = e0.elapsed_time(e1)
            return {"value": c.s * n / (ms / 1e3), "converged": st.status == P.PINT_OK,
                    "status": st.status, "ms": ms, "outer": st.outer_its,
                    "inner": st.inner_its}
        finally:
            P.pint_operator_destroy(op)

    return measure


def batch_measure(ctx, jobs, opts, work):
    """The GPU measurement of a batch launch shape. jobs: (op, B, B0, Y)
    device tensors as for pint_solve_batch; work: the batch's time steps x
    cells (sum of N s). Per shape: a resident plan, one warm-up run, one run
    timed with CUDA events on the current stream, every Y reset to zero
    before each run; value = work / seconds. A shape the device cannot make
    resident, or a job that does not converge, counts as not converged."""
    import torch

    import paper_2504_02117_gb300 as P

    def reset():
        for _, _, _, Y in jobs:
            Y.zero_()

    def measure(shape: BatchShape) -> dict:
        try:
            plan = P.BatchPlan(ctx, jobs, opts, cluster_ctas=shape.cluster_ctas,
                               cta_threads=shape.cta_threads)
        except P.PintError as err:
            return {"value": 0.0, "converged": False, "status": err.code, "error": str(err)}
        try:
            reset()
            plan.run()
            reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            sts = plan.run()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ok = all(x.status == P.PINT_OK for x in sts)
            return {"value": work / (ms / 1e3), "converged": ok, "ms": ms,
                    "inner": sum(x.inner_its for x in sts), "shape": plan.shape()}
        finally:
            plan.close()

    return measure
