"""GPU parity of the linear slab solve (Eq. matrix-fixed-point-equation with
block GMRES inner solves) against the oracle's plain definition: sequential
one-step-at-a-time implicit Euler. FP64 bar: relative 1e-10 per column with
both sides at relative residual 1e-13. Mixed precision bar: 1e-8 after
float64 refinement."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import coupling, fv, krylov, slab

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _setup(P, ctx, dims, s, tau, seed=1, v=(1.0, 0.5, 0.0), lognormal=True, form="grid"):
    """form "grid": the FV constructor (stencil-form SpMM, row-of-tiles ILU(0));
    "csr": the same matrix through pint_operator_assemble (SELL-32 SpMM,
    level-scheduled ILU(0))."""
    n = int(np.prod(dims))
    D = np.exp(synth.normal(seed, n)).reshape(dims[::-1]) if lognormal else \
        np.ones(dims[::-1])
    K = fv.convdiff_matrix(dims, D, v)
    if form == "grid":
        op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), v)
    else:
        Kc = K.tocsr()
        Kc.sort_indices()
        op = P.pint_operator_assemble(ctx, n, Kc.indptr.astype(np.int32),
                                      Kc.indices.astype(np.int32), Kc.data)
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    P.pint_set_coupling(ctx, op, A1, A2)
    B = synth.uniform(seed + 100, n * s).reshape(n, s)
    return op, K, n, A, A1, A2, B


def _colerr(Y, Yref):
    return np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)


@pytest.mark.parametrize("s", [1, 2, 4, 7])
def test_slab_jacobi_2d_config1_shape(P, ctx, s):
    """2-D conv.-diffusion 64x64, D=1, v=(1,0.5), implicit Euler tau=1e-3,
    block GMRES(30) + Jacobi (the 4096-cell workload, s up to 7)."""
    import torch
    op, K, n, A, A1, A2, B = _setup(P, ctx, (64, 64, 1), s, 1e-3, lognormal=False)
    try:
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-13
        o.precond = P.PINT_PC_JACOBI
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-10), err
        # the oracle's own method with the same settings needs a similar effort
        Yo, info = slab.slab_solve(K, np.ones(n), A1, A2, B, None, tol=1e-13, inner_tol=1e-2,
                                   precond="jacobi")
        assert abs(st.outer_its - info["outer"]) <= 2
        assert st.inner_its <= 1.5 * info["inner"] + 5
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("s", [1, 3, 8])
def test_slab_ilu0_3d(P, ctx, s):
    import torch
    dims = (16, 16, 16)
    op, K, n, A, A1, A2, B = _setup(P, ctx, dims, s, 1e-3, seed=2)
    try:
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-13
        o.precond = P.PINT_PC_ILU0
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-10), err
        assert st.setup_ms >= 0.0 and st.inner_its > 0
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("form", ["grid", "csr"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("pc", ["jacobi", "ilu0"])
def test_slab_mixed_precision_refinement(P, ctx, prec, pc, form):
    import torch
    dims = (16, 16, 16)
    s = 4
    op, K, n, A, A1, A2, B = _setup(P, ctx, dims, s, 1e-3, seed=3, form=form)
    try:
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-2
        o.precond = P.PINT_PC_ILU0 if pc == "ilu0" else P.PINT_PC_JACOBI
        o.precision = P.PINT_FP32 if prec == "fp32" else P.PINT_BF16
        P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-8), err
    finally:
        P.pint_operator_destroy(op)


def test_slab_with_b0_and_theta_method(P, ctx):
    """Crank-Nicolson (theta = 1/2) slab after eliminating the explicit stage,
    B0 = M y^n / tau - (1-theta)(K y^n - b^n) (Example ex:time-stepping-matrices)."""
    import torch
    dims = (20, 17, 1)
    n = int(np.prod(dims))
    D = np.exp(0.5 * synth.normal(5, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, -0.5, 0.0))
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, -0.5, 0.0))
    try:
        th, tau, s = 0.5, 2e-3, 5
        A, _, _ = coupling.theta_method(th)
        A1, A2, e = coupling.multistep_matrices(A, s, tau, eliminate_first=True)
        P.pint_set_coupling(ctx, op, A1, A2)
        y0 = synth.uniform(50, n)
        b = synth.uniform(51, n * (s + 1)).reshape(n, s + 1)     # b(t^0..t^s)
        B = b[:, 1:]
        B0 = np.zeros((n, s))
        B0[:, 0] = y0 / tau + e[0] * (b[:, 0] - K @ y0)
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-13
        P.pint_solve_block(ctx, op, _dev(B), _dev(B0), Y, o, raise_on_nonconvergence=True)
        Bst = np.zeros((n, 2 * s))
        Bst[:, 0::2] = b[:, :-1]
        Bst[:, 1::2] = b[:, 1:]
        Yseq = slab.sequential_dirk_linear(K, np.ones(n), A, tau, y0, Bst)[:, 1::2]
        assert np.all(_colerr(Y.cpu().numpy(), Yseq) < 1e-10)
    finally:
        P.pint_operator_destroy(op)


# ------------------------------------------------------------ edge cases
def test_zero_rhs_and_tiny_grid(P, ctx):
    import torch
    op, K, n, A, A1, A2, B = _setup(P, ctx, (3, 3, 1), 3, 1e-2)
    try:
        Y = torch.zeros(n, 3, device="cuda", dtype=torch.float64)
        st = P.pint_solve_block(ctx, op, None, None, Y, raise_on_nonconvergence=True)
        assert st.outer_its == 0 and torch.count_nonzero(Y) == 0
        o = P.pint_opts_default()
        o.tol = 1e-13
        P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-2, np.zeros(n), B)
        assert np.all(_colerr(Y.cpu().numpy(), Yref) < 1e-10)
    finally:
        P.pint_operator_destroy(op)


def test_duplicate_rhs_columns_deflate(P, ctx):
    """Identical right-hand sides of a block-diagonal coupling make the block
    Krylov basis rank deficient: CholQR deflates instead of producing NaN."""
    import torch
    dims = (12, 12, 1)
    n = 144
    D = np.ones(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, 0.5, 0.0))
    try:
        s, tau = 4, 1e-2
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        b = synth.uniform(9, n)
        B = np.column_stack([b, 2 * b, b, -b])
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        assert st.deflations > 0
        y = sp.linalg.spsolve((sp.identity(n) / tau + K).tocsc(), b)
        np.testing.assert_allclose(Y.cpu().numpy(), np.column_stack([y, 2 * y, y, -y]),
                                   rtol=1e-9, atol=1e-12)
    finally:
        P.pint_operator_destroy(op)


def test_nonfinite_rhs_is_breakdown(P, ctx):
    import torch
    op, K, n, A, A1, A2, B = _setup(P, ctx, (10, 10, 1), 2, 1e-2)
    try:
        B[5, 1] = np.nan
        Y = torch.zeros(n, 2, device="cuda", dtype=torch.float64)
        with pytest.raises(P.PintError) as ei:
            P.pint_solve_block(ctx, op, _dev(B), None, Y)
        assert ei.value.code == P.PINT_ERR_BREAKDOWN
    finally:
        P.pint_operator_destroy(op)


def test_iteration_limit_reports_not_converged(P, ctx):
    import torch
    op, K, n, A, A1, A2, B = _setup(P, ctx, (16, 16, 1), 4, 1e-3)
    try:
        Y = torch.zeros(n, 4, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.max_outer = 1
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o)
        assert st.status == P.PINT_ERR_NOT_CONVERGED and st.outer_its == 1
        assert max(st.col_relres[:4]) > o.tol
    finally:
        P.pint_operator_destroy(op)


def test_budget_exceeded_is_nomem(P):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.pint_create(0, 1 << 20)          # 1 MiB budget
    try:
        D = np.ones(64 ** 3)
        with pytest.raises(P.PintError) as ei:
            P.pint_fv_convdiff(c, 64, 64, 64, D, (1.0, 0.0, 0.0))
        assert ei.value.code == P.PINT_ERR_NOMEM
        assert P.pint_bytes_in_use(c) <= 1 << 20
    finally:
        P.pint_destroy(c)


@pytest.mark.parametrize("prec,pc", [("fp64", "ilu0"), ("fp64", "jacobi"), ("fp32", "ilu0"),
                                     ("fp32", "jacobi")])
@pytest.mark.parametrize("s", [1, 3, 8])
def test_slab_block_cg_symmetric_operator(P, ctx, prec, pc, s):
    """Pure diffusion (symmetric J = M/tau + K): the slab with block CG inner
    solves equals sequential stepping, with an effort close to the oracle's
    block CG."""
    import torch
    dims = (12, 10, 9)
    op, K, n, A, A1, A2, B = _setup(P, ctx, dims, s, 1e-3, v=(0.0, 0.0, 0.0))
    try:
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-2 if s > 1 else 1e-6
        o.precond = P.PINT_PC_ILU0 if pc == "ilu0" else P.PINT_PC_JACOBI
        o.precision = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
        o.solver = P.PINT_SOLVER_CG
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-9), err
        Yo, info = slab.slab_solve(K, np.ones(n), A1, A2, B, None, tol=1e-12,
                                   inner_tol=o.inner_tol, precond=pc, solver="cg")
        assert abs(st.outer_its - info["outer"]) <= 2
        assert st.inner_its <= 1.5 * info["inner"] + 5
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("prec,pc", [("fp64", "ilu0"), ("fp64", "jacobi"), ("fp32", "ilu0"),
                                     ("fp32", "jacobi"), ("fp64", "none")])
@pytest.mark.parametrize("s", [1, 3, 8])
def test_slab_block_bicgstab_nonsymmetric_operator(P, ctx, prec, pc, s):
    """Convection-dominated J (upwind, nonsymmetric): the slab with block
    BiCGStab inner solves (the paper's solver for this problem, Sec. 4.1)
    equals sequential stepping, with an effort close to the oracle's block
    BiCGStab."""
    import torch
    dims = (12, 10, 9)
    op, K, n, A, A1, A2, B = _setup(P, ctx, dims, s, 1e-3, v=(20.0, 10.0, 5.0))
    try:
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-2 if s > 1 else 1e-6
        o.precond = {"ilu0": P.PINT_PC_ILU0, "jacobi": P.PINT_PC_JACOBI,
                     "none": P.PINT_PC_NONE}[pc]
        o.precision = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
        o.solver = P.PINT_SOLVER_BICGSTAB
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-9), err
        Yo, info = slab.slab_solve(K, np.ones(n), A1, A2, B, None, tol=1e-12,
                                   inner_tol=o.inner_tol, precond=pc, solver="bicgstab")
        assert abs(st.outer_its - info["outer"]) <= 2
        assert st.inner_its <= 1.5 * info["inner"] + 5
    finally:
        P.pint_operator_destroy(op)


def test_block_bicgstab_dependent_and_zero_columns(P, ctx):
    """Dependent and zero right-hand sides leave the block BiCGStab block at
    the start (CholQR2 deflation) instead of making Rt^T V singular."""
    import torch
    dims = (12, 12, 1)
    n = 144
    D = np.ones(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (20.0, 10.0, 0.0))
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (20.0, 10.0, 0.0))
    try:
        s, tau = 4, 1e-2
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        b = synth.uniform(9, n)
        B = np.column_stack([b, 2 * b, np.zeros(n), -b])
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.precond = P.PINT_PC_ILU0
        o.solver = P.PINT_SOLVER_BICGSTAB
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        assert st.deflations > 0
        y = sp.linalg.spsolve((sp.identity(n) / tau + K).tocsc(), b)
        np.testing.assert_allclose(Y.cpu().numpy(), np.column_stack([y, 2 * y, 0 * y, -y]),
                                   rtol=1e-9, atol=1e-12)
    finally:
        P.pint_operator_destroy(op)


def test_solver_option_is_validated(P, ctx):
    import torch
    op, K, n, A, A1, A2, B = _setup(P, ctx, (6, 5, 1), 2, 1e-2)
    try:
        Y = torch.zeros(n, 2, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.solver = 7
        with pytest.raises(P.PintError) as ei:
            P.pint_solve_block(ctx, op, _dev(B), None, Y, o)
        assert ei.value.code == P.PINT_ERR_INVALID
        o.solver = P.PINT_SOLVER_BICGSTAB
        o.restart = 4                          # nine work blocks need restart >= 8
        with pytest.raises(P.PintError) as ei:
            P.pint_solve_block(ctx, op, _dev(B), None, Y, o)
        assert ei.value.code == P.PINT_ERR_INVALID
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("pc", ["none", "jacobi", "ilu0"])
@pytest.mark.parametrize("s", [4, 8])
def test_slab_global_gmres_equals_sequential_stepping(P, ctx, pc, s):
    """Global GMRES on the unsplit operator (pint_opts.solver =
    PINT_SOLVER_GLOBAL): every column equals sequential implicit Euler to
    1e-10 (FP64, tol 1e-13), and the Arnoldi steps equal the oracle's global
    GMRES on the same problem (up to one step of rounding)."""
    import torch
    dims = (16, 16, 16)
    op, K, n, A, A1, A2, B = _setup(P, ctx, dims, s, 1e-3, seed=7)
    try:
        o = P.pint_opts_default()
        o.tol = 1e-13
        o.precision = P.PINT_FP64
        o.solver = P.PINT_SOLVER_GLOBAL
        o.precond = {"none": P.PINT_PC_NONE, "jacobi": P.PINT_PC_JACOBI, "ilu0": P.PINT_PC_ILU0}[pc]
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        st = P.pint_solve_block(ctx, op, _dev(B), None, Y, o, raise_on_nonconvergence=True)
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
        err = _colerr(Y.cpu().numpy(), Yref)
        assert np.all(err < 1e-10), err
        _, info = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-13, precond=pc,
                                         restart=30)
        assert abs(st.inner_its - info["inner"]) <= 1 + info["cycles"], (st.inner_its, info)
    finally:
        P.pint_operator_destroy(op)


def test_slab_global_gmres_tiny_grid_with_b0_against_dense(P, ctx):
    import torch
    dims = (4, 3, 2)
    n, s = 24, 3
    D = np.exp(synth.normal(21, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.25))
    A, _, _ = coupling.theta_method(0.5)
    A1, A2, e = coupling.multistep_matrices(A, s, 1e-2, eliminate_first=True)
    B = synth.uniform(22, n * s).reshape(n, s)
    B0 = synth.uniform(23, n * s).reshape(n, s)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, 0.5, 0.25))
    try:
        P.pint_set_coupling(ctx, op, A1, A2)
        o = P.pint_opts_default()
        o.tol = 1e-13
        o.precision = P.PINT_FP64
        o.solver = P.PINT_SOLVER_GLOBAL
        o.precond = P.PINT_PC_ILU0
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        P.pint_solve_block(ctx, op, _dev(B), _dev(B0), Y, o, raise_on_nonconvergence=True)
        Yd = slab.solve_all_at_once_dense(K, np.ones(n), A1, A2, B, B0)
        assert np.all(_colerr(Y.cpu().numpy(), Yd) < 1e-10)
        o.precision = P.PINT_FP32
        with pytest.raises(P.PintError) as ei:
            P.pint_solve_block(ctx, op, _dev(B), _dev(B0), Y, o)
        assert ei.value.code == P.PINT_ERR_INVALID
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("s", [2, 4])
def test_fused_update_gram_equals_the_separate_launches(P, s):
    """Block CGS2 with the first update fused into the second Gram pass (the
    default for float32 inner solves at s <= 4) gives bitwise the solution
    and the step counts of the two separate launches (a context created with
    PINT_GRAM_FUSE=0), on the bulk Gram path (a grid operator, 24^3)."""
    import os
    import torch
    out = []
    for fuse in ("1", "0"):
        os.environ["PINT_GRAM_FUSE"] = fuse
        try:
            c = P.pint_create(0)
        finally:
            os.environ.pop("PINT_GRAM_FUSE", None)
        try:
            op, K, n, A, A1, A2, B = _setup(P, c, (24, 24, 24), s, 1e-3, seed=41)
            try:
                o = P.pint_opts_default()
                o.precision = P.PINT_FP32
                o.precond = P.PINT_PC_ILU0
                Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
                st = P.pint_solve_block(c, op, _dev(B), None, Y, o,
                                        raise_on_nonconvergence=True)
                out.append((Y.cpu().numpy(), st.inner_its, st.outer_its))
            finally:
                P.pint_operator_destroy(op)
        finally:
            P.pint_destroy(c)
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]
