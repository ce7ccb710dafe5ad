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
