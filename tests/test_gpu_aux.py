"""Auxiliary subsystems on the GPU: the per-column residual history of a
solve, NVTX ranges per kernel family, and the checked build whose matrix
index gathers record a bad index instead of using it."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import synth
from oracle import coupling, fv, slab

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _slab(P, ctx, dims=(12, 10, 8), s=4, seed=300):
    n = int(np.prod(dims))
    D = np.exp(synth.normal(seed, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, 0.5, 0.0))
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, 1e-3)
    P.pint_set_coupling(ctx, op, A1, A2)
    B = synth.uniform(seed + 1, n * s).reshape(n, s)
    return op, K, n, A1, A2, B


@pytest.mark.parametrize("solver", ["gmres", "global"])
def test_residual_history_of_a_slab_solve(P, ctx, solver):
    """One row per outer iteration: the first is ||F_k|| / ||F_k|| = 1 (Y = 0),
    the last is the stats' final residual and meets tol; for global GMRES the
    row count equals the oracle's outer iterations + 1 (same method)."""
    import torch
    op, K, n, A1, A2, B = _slab(P, ctx)
    try:
        o = P.pint_opts_default()
        o.tol = 1e-10
        o.precision = P.PINT_FP64
        if solver == "global":
            o.solver = P.PINT_SOLVER_GLOBAL
        Y = torch.zeros(n, 4, device="cuda", dtype=torch.float64)
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        h = P.pint_residual_history(ctx)
        assert h.shape == (st.outer_its + 1, 4)
        np.testing.assert_allclose(h[0], 1.0, rtol=1e-12)
        np.testing.assert_array_equal(h[-1], st.as_dict(4)["col_relres"])
        assert np.all(h[-1] <= 1e-10)
        if solver == "global":
            _, info = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-10,
                                             precond="jacobi", restart=30)
            assert h.shape[0] == len(info["history"])
        P.pint_residual_history_reset(ctx)
        assert P.pint_residual_history(ctx).shape[0] == 0
    finally:
        P.pint_operator_destroy(op)


def test_nvtx_ranges_change_nothing(P, ctx):
    """With NVTX ranges on (profiler flag 2, alone or with event timing) the
    solve gives bitwise the same result; flags outside 0..3 are refused."""
    import torch
    op, K, n, A1, A2, B = _slab(P, ctx, seed=310)
    try:
        o = P.pint_opts_default()
        o.precision = P.PINT_FP64
        Ys = []
        for on, nvtx in ((False, False), (False, True), (True, True)):
            P.pint_profile_enable(ctx, on, nvtx=nvtx)
            Y = torch.zeros(n, 4, device="cuda", dtype=torch.float64)
            P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
            Ys.append(Y.cpu().numpy())
        P.pint_profile_enable(ctx, False)
        assert np.array_equal(Ys[0], Ys[1]) and np.array_equal(Ys[0], Ys[2])
        assert P.lib.pint_profile_enable(ctx, 4) == P.PINT_ERR_INVALID
    finally:
        P.pint_operator_destroy(op)


def test_normal_build_reports_no_checks(P, ctx):
    assert P.pint_bounds_report(ctx)[0] == -1


_CHECKED = textwrap.dedent("""
    import sys, json
    sys.path.insert(0, sys.argv[1])
    import numpy as np, torch
    import paper_2504_02117_gb300 as P
    import synth
    from oracle import fv, coupling
    assert P.LIB_PATH.endswith("libpint_bounds.so"), P.LIB_PATH
    ctx = P.pint_create(0)
    out = {}
    out["start"] = P.pint_bounds_report(ctx)
    dims, s = (10, 9, 7), 4
    n = 630
    D = np.exp(synth.normal(320, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0)).tocsr()
    K.sort_indices()
    # a user CSR operator: the SELL SpMM and the coupled residual gather
    op = P.pint_operator_assemble(ctx, n, K.indptr.astype(np.int32),
                                  K.indices.astype(np.int32), K.data)
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, 1e-3)
    P.pint_set_coupling(ctx, op, A1, A2)
    B = torch.tensor(synth.uniform(321, n * s).reshape(n, s), device="cuda")
    o = P.pint_opts_default()
    o.precision = P.PINT_FP64
    Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
    st = P.pint_solve_block(ctx, op, B, None, Y, o, raise_on_nonconvergence=True)
    Yb = torch.zeros(n, s, device="cuda", dtype=torch.float64)
    P.pint_solve_batch(ctx, [(op, B, None, Yb)], o, raise_on_nonconvergence=True)
    out["after_solves"] = P.pint_bounds_report(ctx)
    out["Y"] = Y.cpu().numpy().ravel()[:8].tolist()
    P.pint_test_bounds(ctx, 5, 4)
    out["planted"] = P.pint_bounds_report(ctx)
    P.pint_test_bounds(ctx, 3, 4)
    out["in_range"] = P.pint_bounds_report(ctx)
    P.pint_operator_destroy(op)
    P.pint_destroy(ctx)
    print(json.dumps(out))
""")


def test_checked_build_records_and_skips_a_bad_index():
    """The checked build (libpint_bounds.so, loaded through PINT_LIB in a
    child process): a slab solve and a batched solve on a user CSR operator
    record no bad index; the test entry's out-of-range check (index 5 against
    4, site 99; nothing is accessed through it) is recorded with its site,
    index and bound, and an in-range check is not."""
    import importlib.util
    import json
    spec = importlib.util.spec_from_file_location(
        "pint_build", os.path.join(ROOT, "paper_2504_02117_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = b.build(bounds=True)
    env = dict(os.environ, PINT_LIB=lib)
    r = subprocess.run([sys.executable, "-c", _CHECKED, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["start"][0] == 0
    assert out["after_solves"][0] == 0, out
    assert out["planted"] == [1, 99, 5, 4], out
    assert out["in_range"][0] == 0, out
