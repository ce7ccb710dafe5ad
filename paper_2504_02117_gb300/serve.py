"""Continuous-batching request loop for time-slab solves on one GPU.

Requests (linear convection-diffusion slabs of s coupled implicit-Euler
steps on n^3 cells, float32 or float64 inner solves) arrive on their own
clock. The dispatcher admits them in arrival order as soon as a slot is free
and their device memory fits the budget; each slot is a worker thread with
its own library context and CUDA stream, so admitted solves run concurrently
on the device while later requests keep arriving (the library's calls
release the interpreter lock). A request whose estimate exceeds the whole
budget is rejected, never queued forever.

With the batch lane on, small float64 requests (N s up to batch_max_unknowns)
need no slot: once admitted by memory they wait in the lane, and the lane's
worker solves every waiting request in ONE launch of the batched persistent
kernel (pint_solve_batch: a cluster of CTAs per request, a device job queue,
global GMRES + Jacobi). Requests that arrive while a batch runs form the
next batch, so the lane batches continuously at launch granularity while the
slots keep serving the larger and the float32 requests beside it.

The solve itself is a callable (slot, request) -> dict, so the admission
logic can be exercised without a GPU.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time
from typing import Callable, Optional


@dataclasses.dataclass
class SlabRequest:
    rid: int
    arrival: float                 # seconds after the stream starts
    dims: tuple                    # (nx, ny, nz)
    s: int
    precision: str = "fp32"        # inner solve: "fp32" or "fp64"
    D: object = None               # host diffusion field (nz, ny, nx)
    B: object = None               # host right-hand side block (N x s)
    velocity: tuple = (1.0, 0.5, 0.0)
    tau: float = 1e-3
    tol: float = 1e-10
    inner_tol: float = 1e-2
    restart: int = 30
    solver: str = "gmres"          # inner solver: "gmres", "cg" or "bicgstab"
    # filled by the server
    admitted: Optional[float] = None
    finished: Optional[float] = None
    slot: Optional[int] = None
    status: Optional[int] = None
    outer: Optional[int] = None
    inner: Optional[int] = None
    Y: object = None
    error: Optional[str] = None

    @property
    def cells(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])


def estimate_batch_bytes(cells: int, s: int, restart: int = 30) -> int:
    """Device bytes one request holds in the batch lane: its operator (about
    440 bytes per cell), B and Y, and one cluster workspace of (restart + 3)
    N s + 8 N doubles (an upper bound: a launch holds one workspace per
    resident cluster), plus 25 % slack."""
    b = 440 * cells + 16 * cells * s + 8 * ((restart + 3) * cells * s + 8 * cells)
    return int(1.25 * b)


def estimate_bytes(cells: int, s: int, precision: str, restart: int = 30) -> int:
    """Device bytes one slab solve holds: the operator (CSR, SELL, float64 and
    float32 inner values, ILU(0) factors and stencil coefficients, about 440
    bytes per cell for a 7-point stencil), the Krylov basis and work blocks,
    the float64 residual blocks and the caller's B and Y, plus 25 % slack."""
    es = 8 if precision == "fp64" else 4
    n_pad = -(-cells // 64) * 64
    b = 440 * cells + (restart + 4) * n_pad * s * es + 48 * cells * s + (64 << 20)
    return int(1.25 * b)


class SlabServer:
    def __init__(self, slots: int = 4, hbm_budget: Optional[int] = None, device: int = 0,
                 solve: Optional[Callable] = None, keep_results: bool = False,
                 batch_lane: bool = False, batch_max_unknowns: int = 1 << 19,
                 batch_max_jobs: int = 512, solve_batch: Optional[Callable] = None,
                 batch_cluster: int = 8, batch_threads: int = 512):
        self.slots = slots
        self.device = device
        self.keep = keep_results
        self._solve = solve or self._gpu_solve
        self.batch_lane = batch_lane
        self.batch_max_unknowns = int(batch_max_unknowns)
        self.batch_max_jobs = int(batch_max_jobs)
        self._solve_batch = solve_batch or self._gpu_solve_batch
        # one launch shape for every batch: a request's result then does not
        # depend on which batch it joined (fixed reduction order)
        self.batch_cluster = int(batch_cluster)
        self.batch_threads = int(batch_threads)
        self._bctx = None
        self._bstream = None
        if hbm_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.8 * free)
        self.budget = int(hbm_budget)
        self._ctx = [None] * slots
        self._stream = [None] * slots

    # --------------------------------------------------------- GPU solve
    def _gpu_solve(self, slot: int, r: SlabRequest) -> dict:
        import numpy as np
        import torch
        import paper_2504_02117_gb300 as P
        if self._ctx[slot] is None:
            torch.cuda.set_device(self.device)
            self._ctx[slot] = P.pint_create(self.device)
            self._stream[slot] = torch.cuda.Stream(self.device)
        ctx, st = self._ctx[slot], self._stream[slot]
        s = r.s
        with torch.cuda.stream(st):
            op = P.pint_fv_convdiff(ctx, *r.dims, np.ascontiguousarray(r.D).ravel(), r.velocity,
                                    stream=st)
            try:
                P.pint_set_coupling(ctx, op, (np.eye(s) - np.eye(s, k=-1)) / r.tau, np.eye(s))
                Bd = torch.as_tensor(np.ascontiguousarray(r.B), dtype=torch.float64).to(
                    f"cuda:{self.device}")
                Y = torch.zeros(r.cells, s, device=f"cuda:{self.device}", dtype=torch.float64)
                o = P.pint_opts_default()
                o.tol = r.tol
                o.inner_tol = r.inner_tol
                o.restart = r.restart
                o.precond = P.PINT_PC_ILU0
                o.precision = P.PINT_FP64 if r.precision == "fp64" else P.PINT_FP32
                o.solver = {"gmres": P.PINT_SOLVER_GMRES, "cg": P.PINT_SOLVER_CG,
                            "bicgstab": P.PINT_SOLVER_BICGSTAB}[r.solver]
                res = P.pint_solve_block(ctx, op, Bd, None, Y, o, stream=st)
                out = {"status": res.status, "outer": res.outer_its, "inner": res.inner_its}
                if self.keep:
                    out["Y"] = Y.cpu().numpy()
                st.synchronize()
            finally:
                P.pint_operator_destroy(op)
        return out

    def batchable(self, r: SlabRequest) -> bool:
        return (self.batch_lane and r.precision == "fp64" and r.solver == "gmres"
                and r.restart <= 32 and r.cells * r.s <= self.batch_max_unknowns)

    def need_bytes(self, r: SlabRequest) -> int:
        if self.batchable(r):
            return estimate_batch_bytes(r.cells, r.s, r.restart)
        return estimate_bytes(r.cells, r.s, r.precision, r.restart)

    def _gpu_solve_batch(self, reqs: list) -> list:
        """One launch of the batched kernel for every request of the batch."""
        import numpy as np
        import torch
        import paper_2504_02117_gb300 as P
        if self._bctx is None:
            torch.cuda.set_device(self.device)
            self._bctx = P.pint_create(self.device)
            self._bstream = torch.cuda.Stream(self.device)
        ctx, st = self._bctx, self._bstream
        dev = f"cuda:{self.device}"
        ops, jobs, Ys = [], [], []
        with torch.cuda.stream(st):
            try:
                for r in reqs:
                    op = P.pint_fv_convdiff(ctx, *r.dims, np.ascontiguousarray(r.D).ravel(),
                                            r.velocity, stream=st)
                    ops.append(op)
                    P.pint_set_coupling(ctx, op, (np.eye(r.s) - np.eye(r.s, k=-1)) / r.tau,
                                        np.eye(r.s))
                    Bd = torch.as_tensor(np.ascontiguousarray(r.B), dtype=torch.float64).to(dev)
                    Y = torch.zeros(r.cells, r.s, device=dev, dtype=torch.float64)
                    jobs.append((op, Bd, None, Y))
                    Ys.append(Y)
                o = P.pint_opts_default()
                o.tol = min(r.tol for r in reqs)
                o.restart = max(r.restart for r in reqs)
                o.precond = P.PINT_PC_JACOBI
                o.precision = P.PINT_FP64
                sts = P.pint_solve_batch(ctx, jobs, o, cluster_ctas=self.batch_cluster,
                                         cta_threads=self.batch_threads, stream=st)
                outs = []
                for r, x, Y in zip(reqs, sts, Ys):
                    d = {"status": x.status, "outer": x.outer_its, "inner": x.inner_its}
                    if self.keep:
                        d["Y"] = Y.cpu().numpy()
                    outs.append(d)
                st.synchronize()
            finally:
                for op in ops:
                    P.pint_operator_destroy(op)
        return outs

    def close(self):
        import paper_2504_02117_gb300 as P
        for c in self._ctx:
            if c is not None:
                P.pint_destroy(c)
        self._ctx = [None] * self.slots
        if self._bctx is not None:
            P.pint_destroy(self._bctx)
            self._bctx = None

    # ---------------------------------------------------------- the loop
    def run(self, requests: list) -> dict:
        reqs = sorted(requests, key=lambda r: r.arrival)
        cond = threading.Condition()
        free = list(range(self.slots))[::-1]
        state = {"reserved": 0, "running": 0, "max_running": 0, "peak_reserved": 0,
                 "batches": 0, "batched": 0, "max_batch": 0, "stop": False}
        inbox = [queue.Queue() for _ in range(self.slots)]
        lane = []                                   # admitted batch-lane requests
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def finish(r, out, need, slot=None):
            r.status = out.get("status")
            r.outer = out.get("outer")
            r.inner = out.get("inner")
            r.Y = out.get("Y")
            with cond:
                r.finished = now()
                state["reserved"] -= need
                state["running"] -= 1
                if slot is not None:
                    free.append(slot)
                cond.notify_all()

        def worker(slot):
            while True:
                item = inbox[slot].get()
                if item is None:
                    return
                r, need = item
                try:
                    out = self._solve(slot, r)
                except Exception as e:            # the request fails, the server goes on
                    out = {"status": -1}
                    r.error = str(e)[:300]
                finish(r, out, need, slot)

        def lane_worker():
            while True:
                with cond:
                    while not lane and not state["stop"]:
                        cond.wait()
                    if not lane:
                        return
                    batch = lane[:self.batch_max_jobs]
                    del lane[:len(batch)]
                    state["batches"] += 1
                    state["batched"] += len(batch)
                    state["max_batch"] = max(state["max_batch"], len(batch))
                try:
                    outs = self._solve_batch([r for r, _ in batch])
                except Exception as e:            # the batch fails, the server goes on
                    outs = [{"status": -1}] * len(batch)
                    for r, _ in batch:
                        r.error = str(e)[:300]
                for (r, need), out in zip(batch, outs):
                    finish(r, out, need)

        threads = [threading.Thread(target=worker, args=(i,), daemon=True)
                   for i in range(self.slots)]
        if self.batch_lane:
            threads.append(threading.Thread(target=lane_worker, daemon=True))
        for t in threads:
            t.start()
        pending = list(reqs)
        rejected = []
        try:
            with cond:
                while pending or state["running"]:
                    t = now()
                    # admit in arrival order while the memory fits and, for
                    # requests outside the batch lane, a slot is free
                    while pending and pending[0].arrival <= t:
                        r = pending[0]
                        in_lane = self.batchable(r)
                        if not in_lane and not free:
                            break
                        need = self.need_bytes(r)
                        if need > self.budget:
                            pending.pop(0)
                            r.status, r.error = -2, "larger than the device budget"
                            rejected.append(r)
                            continue
                        if state["reserved"] + need > self.budget:
                            break                   # wait for memory to free up
                        pending.pop(0)
                        r.admitted = t
                        state["reserved"] += need
                        state["running"] += 1
                        state["max_running"] = max(state["max_running"], state["running"])
                        state["peak_reserved"] = max(state["peak_reserved"], state["reserved"])
                        if in_lane:
                            r.slot = "batch"
                            lane.append((r, need))
                            cond.notify_all()
                        else:
                            slot = free.pop()
                            r.slot = slot
                            inbox[slot].put((r, need))
                    if pending and pending[0].arrival > t:
                        cond.wait(timeout=pending[0].arrival - t)
                    elif pending or state["running"]:
                        cond.wait(timeout=0.5)
        finally:
            with cond:
                state["stop"] = True
                cond.notify_all()
            for q in inbox:
                q.put(None)
            for th in threads:
                th.join()
        done = [r for r in reqs if r.finished is not None]
        summ = summarize(done, rejected, state, self.slots, self.budget)
        if self.batch_lane:
            summ.update({"batch_launches": state["batches"], "batched_requests": state["batched"],
                         "max_batch": state["max_batch"],
                         "batch_max_unknowns": self.batch_max_unknowns})
        return summ


def summarize(done: list, rejected: list, state: dict, slots: int, budget: int) -> dict:
    import numpy as np
    ok = [r for r in done if r.status == 0]
    lat = np.array([r.finished - r.arrival for r in done]) if done else np.zeros(0)
    wait = np.array([r.admitted - r.arrival for r in done]) if done else np.zeros(0)
    span = (max(r.finished for r in done) - min(r.arrival for r in done)) if done else 0.0
    work = sum(r.s * r.cells for r in ok)
    pct = (lambda a, q: float(np.percentile(a, q)) if len(a) else None)
    return {"requests": len(done) + len(rejected), "completed": len(ok),
            "failed": len(done) - len(ok), "rejected": len(rejected),
            "p50_latency_s": pct(lat, 50), "p99_latency_s": pct(lat, 99),
            "p50_queue_s": pct(wait, 50), "p99_queue_s": pct(wait, 99),
            "makespan_s": span, "time_step_dof_per_s": work / span if span > 0 else None,
            "slots": slots, "max_concurrent": state["max_running"],
            "budget_bytes": budget, "peak_reserved_bytes": state["peak_reserved"]}
