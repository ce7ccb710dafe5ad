"""GPU parity of the nonlinear pieces (a11) and of Algorithm 1 against the
oracle: the column-wise residual of Eq. matrix-equation-pipelining, the
first-column Jacobian, and whole pipelined runs against sequential Newton
stepping (the plain definition)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import coupling, fv, newton

pytestmark = pytest.mark.gpu

VG = (1.0, 2.0, 0.05, 0.4, 1.0 / 16.0)


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _richards(dims, seed=4):
    n = int(np.prod(dims))
    Ks = np.exp(2.0 * synth.correlated_field(seed, dims[::-1], 2.0))
    vg = fv.VanGenuchten(*VG[:4])
    return n, Ks, vg, newton.RichardsProblem(dims, Ks, vg, VG[4])


def _make(P, ctx, kind, dims):
    if kind == "diffreact":
        prob = P.pint_problem_create(ctx, P.PINT_PROBLEM_DIFFREACT, *dims)
        return prob, newton.DiffReactProblem(dims), int(np.prod(dims))
    n, Ks, vg, oprob = _richards(dims)
    prob = P.pint_problem_create(ctx, P.PINT_PROBLEM_RICHARDS, *dims, params=VG,
                                 field=_dev(Ks.ravel()))
    return prob, oprob, n


def _state(kind, dims, n, s, seed):
    if kind == "diffreact":
        return 0.5 + 0.4 * synth.uniform(seed, n * s).reshape(n, s)
    z, _ = fv.richards_cells(dims)
    return (-z - 0.5)[:, None] + 0.3 * synth.uniform(seed, n * s).reshape(n, s)


@pytest.mark.parametrize("kind,dims", [("diffreact", (17, 13, 1)), ("richards", (7, 6, 5))])
@pytest.mark.parametrize("s,tab,g0", [(2, "sdirk2", 1), (4, "ie", 0), (3, "sdirk2", 2),
                                      (16, "ie", 5)])
def test_window_residual_matches_oracle(P, ctx, kind, dims, s, tab, g0):
    import torch
    prob, oprob, n = _make(P, ctx, kind, dims)
    try:
        A, _, c = coupling.sdirk2() if tab == "sdirk2" else coupling.implicit_euler()
        tau = 0.01
        A1, A2, terms, times = coupling.window_matrices(A, c, tau, g0, s)
        op = P.pint_problem_operator(prob)
        P.pint_set_coupling(ctx, op, A1, A2)
        Y = _state(kind, dims, n, s, 3)
        B0 = synth.uniform(4, n * s).reshape(n, s)
        R = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_problem_residual(ctx, prob, times, _dev(Y), _dev(B0), R)
        ref = newton.window_residual(oprob, A1, A2, times, Y, B0)
        h2 = float(dims[0]) ** 2
        np.testing.assert_allclose(R.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * h2 * 40)
    finally:
        P.pint_problem_destroy(prob)


@pytest.mark.parametrize("kind,dims", [("diffreact", (17, 13, 1)), ("richards", (7, 6, 5))])
def test_eval_and_jacobian_match_oracle(P, ctx, kind, dims):
    import torch
    prob, oprob, n = _make(P, ctx, kind, dims)
    try:
        t = 0.03
        y = _state(kind, dims, n, 1, 5)[:, 0]
        m = torch.empty(n, device="cuda", dtype=torch.float64)
        f = torch.empty(n, device="cuda", dtype=torch.float64)
        P.pint_problem_eval(ctx, prob, t, _dev(y), m, f)
        h2 = float(dims[0]) ** 2
        np.testing.assert_allclose(m.cpu().numpy(), oprob.mass(y), rtol=1e-13)
        np.testing.assert_allclose(f.cpu().numpy(), oprob.f(t, y), rtol=1e-12, atol=1e-12 * h2)
        # Jacobian through one Newton step: afterwards the operator holds
        # J = alpha M'(Y_0) + beta Df(t_0, Y_0), checked by applying it
        s, tau = 2, 0.01
        A, _, c = coupling.sdirk2()
        A1, A2, terms, times = coupling.window_matrices(A, c, tau, 0, s)
        op = P.pint_problem_operator(prob)
        P.pint_set_coupling(ctx, op, A1, A2)
        Y = np.column_stack([y, y])
        B0 = np.zeros((n, s))
        o = P.pint_opts_default()
        o.tol = 1e-30
        o.inner_tol = 1e-3
        o.precond = P.PINT_PC_JACOBI
        Yd = _dev(Y)
        conv, st = P.pint_newton_step(ctx, prob, times, Yd, _dev(B0), o)
        assert not conv and st.inner_its > 0
        X = synth.uniform(6, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_inner_apply(ctx, op, _dev(X), Z)
        J = sp.diags(A1[0, 0] * oprob.dmass(y)) + A2[0, 0] * oprob.jac(times[0], y)
        np.testing.assert_allclose(Z.cpu().numpy(), J @ X, rtol=1e-11, atol=1e-11 * h2)
    finally:
        P.pint_problem_destroy(prob)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipeline_diffreact_equals_sequential(P, ctx, prec):
    import torch
    dims = (16, 16, 1)
    prob, oprob, n = _make(P, ctx, "diffreact", dims)
    try:
        A, _, c = coupling.sdirk2()
        tau, G, s = 0.01, 8, 2
        y0 = np.full(n, 0.5)
        out = torch.zeros(n, G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-5 if prec == "fp64" else 1e-4
        o.precond = P.PINT_PC_ILU0
        o.precision = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
        o.max_outer = 40
        st = P.pint_pipeline_run(ctx, prob, A, c, tau, s, _dev(y0), G, out, o)
        Yseq, _ = newton.sequential_dirk_newton(oprob, A, c, tau, y0, G)
        err = np.linalg.norm(out.cpu().numpy() - Yseq, axis=0) / np.linalg.norm(Yseq, axis=0)
        assert np.all(err < (1e-10 if prec == "fp64" else 1e-8)), err
        assert st.outer_its >= G
    finally:
        P.pint_problem_destroy(prob)


def test_pipeline_richards_equals_sequential(P, ctx):
    import torch
    dims = (8, 8, 8)
    prob, oprob, n = _make(P, ctx, "richards", dims)
    try:
        A, _, c = coupling.implicit_euler()
        tau, G, s = 1.0 / 96.0, 6, 4
        z, _ = fv.richards_cells(dims)
        y0 = -z
        out = torch.zeros(n, G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-6
        o.precond = P.PINT_PC_ILU0
        o.max_outer = 60
        o.max_step = 1.0                 # step bound of 1 m of head per Newton update
        P.pint_pipeline_run(ctx, prob, A, c, tau, s, _dev(y0), G, out, o)
        Yseq, _ = newton.sequential_dirk_newton(oprob, A, c, tau, y0, G)
        err = np.linalg.norm(out.cpu().numpy() - Yseq, axis=0) / np.linalg.norm(Yseq, axis=0)
        assert np.all(err < 1e-10), err
    finally:
        P.pint_problem_destroy(prob)


def test_lscheme_matrix_matches_oracle(P, ctx):
    """With opts.lscheme_L < 0 the outer iteration's matrix is the L-scheme
    matrix of Sec. 4.3, alpha L I + beta A(y_0) with L the Lipschitz constant
    of theta and the conductivities frozen at y_0."""
    import torch
    dims = (7, 6, 5)
    prob, oprob, n = _make(P, ctx, "richards", dims)
    try:
        y = _state("richards", dims, n, 1, 5)[:, 0]
        s, tau = 2, 0.01
        A, _, c = coupling.implicit_euler()
        A1, A2, terms, times = coupling.window_matrices(A, c, tau, 0, s)
        op = P.pint_problem_operator(prob)
        P.pint_set_coupling(ctx, op, A1, A2)
        o = P.pint_opts_default()
        o.tol = 1e-30
        o.inner_tol = 1e-3
        o.precond = P.PINT_PC_JACOBI
        o.lscheme_L = -1.0
        conv, st = P.pint_newton_step(ctx, prob, times, _dev(np.column_stack([y, y])),
                                      _dev(np.zeros((n, s))), o)
        assert not conv
        X = synth.uniform(6, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_inner_apply(ctx, op, _dev(X), Z)
        J = newton.linearisation(oprob, A1[0, 0], A2[0, 0], times[0], y,
                                 fv.VanGenuchten(*VG[:4]).lipschitz())
        h2 = float(dims[0]) ** 2
        np.testing.assert_allclose(Z.cpu().numpy(), J @ X, rtol=1e-11, atol=1e-11 * h2)
        # the L-scheme is a Richards option only
        dprob, _, _ = _make(P, ctx, "diffreact", (9, 8, 1))
        try:
            P.pint_set_coupling(ctx, P.pint_problem_operator(dprob), A1, A2)
            with pytest.raises(P.PintError):
                P.pint_newton_step(ctx, dprob, times, _dev(np.full((72, s), 0.5)),
                                   _dev(np.zeros((72, s))), o)
        finally:
            P.pint_problem_destroy(dprob)
    finally:
        P.pint_problem_destroy(prob)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipeline_richards_lscheme_equals_sequential(P, ctx, prec):
    """Algorithm 1 with the L-scheme outer iteration reaches the stages of
    sequential Newton stepping (the plain definition) on 8^3 cells."""
    import torch
    dims = (8, 8, 8)
    prob, oprob, n = _make(P, ctx, "richards", dims)
    try:
        A, _, c = coupling.implicit_euler()
        tau, G, s = 1.0 / 96.0, 6, 4
        z, _ = fv.richards_cells(dims)
        y0 = -z
        out = torch.zeros(n, G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-10
        o.inner_tol = 1e-8 if prec == "fp64" else 1e-5
        o.precond = P.PINT_PC_ILU0
        o.precision = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
        o.max_outer = 150
        o.max_step = 1.0
        o.lscheme_L = -1.0
        P.pint_pipeline_run(ctx, prob, A, c, tau, s, _dev(y0), G, out, o)
        Yseq, _ = newton.sequential_dirk_newton(oprob, A, c, tau, y0, G)
        # ||R_0|| <= 1e-10 ||B0_0|| bounds the stage error by ~1e-7 (see the
        # oracle's own L-scheme test)
        np.testing.assert_allclose(out.cpu().numpy(), Yseq, rtol=0, atol=2e-7)
    finally:
        P.pint_problem_destroy(prob)


def test_pipeline_richards_lscheme_block_cg(P, ctx):
    """The L-scheme matrix is symmetric positive definite (one conductivity
    per face): Algorithm 1 with block CG inner solves reaches the stages of
    sequential Newton stepping on 8^3 cells."""
    import torch
    dims = (8, 8, 8)
    prob, oprob, n = _make(P, ctx, "richards", dims)
    try:
        A, _, c = coupling.implicit_euler()
        tau, G, s = 1.0 / 96.0, 6, 4
        z, _ = fv.richards_cells(dims)
        out = torch.zeros(n, G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-10
        o.inner_tol = 1e-8
        o.precond = P.PINT_PC_ILU0
        o.max_outer = 150
        o.max_step = 1.0
        o.lscheme_L = -1.0
        o.solver = P.PINT_SOLVER_CG
        P.pint_pipeline_run(ctx, prob, A, c, tau, s, _dev(-z), G, out, o)
        Yseq, _ = newton.sequential_dirk_newton(oprob, A, c, tau, -z, G)
        np.testing.assert_allclose(out.cpu().numpy(), Yseq, rtol=0, atol=2e-7)
    finally:
        P.pint_problem_destroy(prob)


def test_pipeline_diffreact_block_bicgstab(P, ctx):
    """Algorithm 1 with block BiCGStab inner solves on the nonsymmetric
    diffusion-reaction Jacobian: the window's identical trailing columns are
    deflated at the start of every inner solve, and the stages equal
    sequential Newton stepping."""
    import torch
    dims = (16, 16, 1)
    prob, oprob, n = _make(P, ctx, "diffreact", dims)
    try:
        A, _, c = coupling.sdirk2()
        tau, G, s = 0.01, 8, 2
        y0 = np.full(n, 0.5)
        out = torch.zeros(n, G, device="cuda", dtype=torch.float64)
        o = P.pint_opts_default()
        o.tol = 1e-12
        o.inner_tol = 1e-5
        o.precond = P.PINT_PC_ILU0
        o.max_outer = 40
        o.solver = P.PINT_SOLVER_BICGSTAB
        st = P.pint_pipeline_run(ctx, prob, A, c, tau, s, _dev(y0), G, out, o)
        Yseq, _ = newton.sequential_dirk_newton(oprob, A, c, tau, y0, G)
        err = np.linalg.norm(out.cpu().numpy() - Yseq, axis=0) / np.linalg.norm(Yseq, axis=0)
        assert np.all(err < 1e-10), err
        assert st.outer_its >= G
    finally:
        P.pint_problem_destroy(prob)
