"""The serving loop on the GPU: requests of mixed grids, block widths and
precisions run concurrently (one context and stream per slot) and each
result is the same alone as in the mix; every result meets the tolerance in
the oracle's float64 residual."""
import numpy as np
import pytest

import synth
from oracle import fv, slab
from paper_2504_02117_gb300 import serve

pytestmark = pytest.mark.gpu


def _req(rid, arrival, n, s, prec):
    w = synth.convdiff_3d(n, s)
    return serve.SlabRequest(rid=rid, arrival=arrival, dims=w.dims, s=s, precision=prec,
                             D=synth.diffusion_field(w), B=synth.rhs_block(w),
                             velocity=w.velocity, tau=w.tau, tol=w.tol, inner_tol=1e-2)


def test_results_are_the_same_alone_and_in_the_mix():
    shapes = [(16, 2, "fp32"), (24, 4, "fp64"), (32, 8, "fp32"), (16, 8, "fp64"),
              (24, 2, "fp32"), (32, 4, "fp64"), (16, 4, "fp32"), (24, 8, "fp32"),
              (32, 2, "fp64"), (16, 16, "fp32")]
    reqs = [_req(i, 0.001 * i, *sh) for i, sh in enumerate(shapes)]
    srv = serve.SlabServer(slots=3, keep_results=True)
    try:
        summ = srv.run(reqs)
    finally:
        srv.close()
    assert summ["completed"] == len(shapes), [r.error for r in reqs]
    assert summ["max_concurrent"] >= 2                     # work overlapped
    alone = serve.SlabServer(slots=1, keep_results=True)
    try:
        for r in reqs[::3]:
            a = _req(100 + r.rid, 0.0, r.dims[0], r.s, r.precision)
            alone.run([a])
            assert a.status == 0
            # deterministic kernels (fixed-order reductions): identical results
            np.testing.assert_array_equal(a.Y, r.Y)
    finally:
        alone.close()
    for r in reqs[:4]:
        K = fv.convdiff_matrix(r.dims, r.D, r.velocity)
        A1 = (np.eye(r.s) - np.eye(r.s, k=-1)) / r.tau
        R = slab.coupled_residual(K, np.ones(r.cells), A1, np.eye(r.s), r.Y, r.B)
        F = slab.rhs_F(np.eye(r.s), r.B)
        assert np.all(np.linalg.norm(R, axis=0) <= r.tol * 1.001 * np.linalg.norm(F, axis=0))


def test_batch_lane_results_are_the_same_alone_and_in_the_mix():
    """With the batch lane on, small float64 requests are solved several per
    launch by the batched kernel (fixed launch shape) beside the slots' float32
    solves: each lane result is bitwise the one it gets alone, meets the
    tolerance in the oracle's float64 residual and equals sequential stepping
    to 1e-8."""
    shapes = [(16, 2, "fp64"), (16, 4, "fp64"), (24, 2, "fp64"), (16, 8, "fp64"),
              (24, 4, "fp32"), (16, 16, "fp64"), (32, 2, "fp64"), (24, 2, "fp32")]
    reqs = [_req(i, 0.0005 * i, *sh) for i, sh in enumerate(shapes)]
    srv = serve.SlabServer(slots=2, keep_results=True, batch_lane=True,
                           batch_max_unknowns=32 ** 3 * 2)
    try:
        summ = srv.run(reqs)
    finally:
        srv.close()
    assert summ["completed"] == len(shapes), [r.error for r in reqs]
    lane = [r for r in reqs if r.slot == "batch"]
    assert len(lane) == 6 and summ["batched_requests"] == 6
    alone = serve.SlabServer(slots=1, keep_results=True, batch_lane=True,
                             batch_max_unknowns=32 ** 3 * 2)
    try:
        for r in lane[::2]:
            a = _req(100 + r.rid, 0.0, r.dims[0], r.s, r.precision)
            alone.run([a])
            assert a.status == 0 and a.slot == "batch"
            np.testing.assert_array_equal(a.Y, r.Y)
    finally:
        alone.close()
    from oracle import coupling
    A, _, _ = coupling.implicit_euler()
    for r in lane:
        K = fv.convdiff_matrix(r.dims, r.D, r.velocity)
        A1 = (np.eye(r.s) - np.eye(r.s, k=-1)) / r.tau
        R = slab.coupled_residual(K, np.ones(r.cells), A1, np.eye(r.s), r.Y, r.B)
        F = slab.rhs_F(np.eye(r.s), r.B)
        assert np.all(np.linalg.norm(R, axis=0) <= r.tol * 1.001 * np.linalg.norm(F, axis=0))
        Yref = slab.sequential_dirk_linear(K, np.ones(r.cells), A, r.tau, np.zeros(r.cells), r.B)
        err = np.linalg.norm(r.Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)
        assert np.all(err < 1e-8), err
