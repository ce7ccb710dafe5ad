"""The autotuner on the GPU: one warm-up and one timed slab solve per
candidate on a 16^3 convection-diffusion operator; every candidate
converges, the ranking follows the measured throughput, and the choice is
cached."""
import numpy as np
import pytest

import synth
from paper_2504_02117_gb300 import tune

pytestmark = pytest.mark.gpu


def test_autotune_slab_width_and_solver(P, ctx, tmp_path):
    dims = (16, 16, 16)
    n = 16 ** 3
    D = np.exp(synth.normal(3, n))
    measure = tune.slab_measure(ctx, dims, D, (1.0, 0.5, 0.0), 1e-3,
                                lambda s: synth.uniform(40 + s, n * s).reshape(n, s))
    cands = tune.grid((1, 2, 4), ("gmres", "bicgstab"), ("fp32",))
    best, table = tune.autotune(measure, cands, repeats=2)
    assert best in cands
    assert all(e["converged"] for e in table), [e["last"] for e in table]
    vals = [e["value"] for e in table]
    assert vals == sorted(vals, reverse=True) and vals[0] > 0.0
    cache = tune.TuneCache(str(tmp_path / "tune.json"))
    op = P.pint_fv_convdiff(ctx, *dims, D, (1.0, 0.5, 0.0))
    try:
        nnz = P.pint_operator_nnz(op)
    finally:
        P.pint_operator_destroy(op)
    key = tune.TuneCache.key(dims, nnz, "ilu0", 1e-10, "gpu0")
    cache.put(key, best, table[0]["value"])
    assert tune.TuneCache(cache.path).get(key) == best


def test_autotune_batch_launch_shape(P, ctx, tmp_path):
    """The batched kernel's launch shape measured on a batch of 40 uneven
    2-D slabs: every shape converges, the ranking follows the measured
    throughput, and the choice is cached under the batch's key."""
    import torch
    from oracle import coupling
    A, _, _ = coupling.implicit_euler()
    ops, jobs, sizes = [], [], []
    try:
        for q in range(40):
            nx = (24, 32, 40)[q % 3]
            s = (2, 4, 8)[q % 3]
            n = nx * nx
            op = P.pint_fv_convdiff(ctx, nx, nx, 1, np.exp(synth.normal(500 + q, n)),
                                    (1.0, 0.5, 0.0))
            ops.append(op)
            A1, A2, _ = coupling.multistep_matrices(A, s, 1e-3)
            P.pint_set_coupling(ctx, op, A1, A2)
            B = torch.tensor(synth.uniform(600 + q, n * s).reshape(n, s), device="cuda")
            jobs.append((op, B, None, torch.zeros(n, s, device="cuda", dtype=torch.float64)))
            sizes.append(n * s)
        o = P.pint_opts_default()
        o.precision = P.PINT_FP64
        measure = tune.batch_measure(ctx, jobs, o, sum(sizes))
        shapes = tune.batch_shapes((1, 2, 4), (512,))
        best, table = tune.autotune(measure, shapes, repeats=2)
        assert best in shapes
        assert all(e["converged"] for e in table), [e["last"] for e in table]
        vals = [e["value"] for e in table]
        assert vals == sorted(vals, reverse=True) and vals[0] > 0.0
        cache = tune.TuneCache(str(tmp_path / "tune.json"))
        key = tune.TuneCache.batch_key(sizes, "gpu0")
        cache.put_batch(key, best, table[0]["value"])
        assert tune.TuneCache(cache.path).get_batch(key) == best
    finally:
        for op in ops:
            P.pint_operator_destroy(op)
