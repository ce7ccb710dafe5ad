"""Pins of oracle.newton: sequential Newton == linear stepping, quadratic
convergence, time orders, Algorithm 1 == sequential stepping (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupling, fv, newton, slab


def _linear(n=4, seed=0):
    dims = (n, n, 1)
    rng = np.random.default_rng(seed)
    D = np.exp(rng.standard_normal(dims[::-1]))
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    Md = 1.0 + 0.5 * rng.random(n * n)
    b1, b2 = rng.standard_normal((2, n * n))
    return K, Md, (lambda t: math.sin(3 * t) * b1 + math.cos(2 * t) * b2), rng


@pytest.mark.parametrize("tab", ["ie", "sdirk2"])
def test_sequential_newton_equals_linear_stepping(tab):
    K, Md, b, rng = _linear()
    A, _, c = coupling.implicit_euler() if tab == "ie" else coupling.sdirk2()
    m = A.shape[0]
    tau, steps = 0.05, 3
    y0 = rng.standard_normal(K.shape[0])
    G = steps * m
    tg = np.array([(g // m + c[g % m]) * tau for g in range(G)])
    Bst = np.column_stack([b(t) for t in tg])
    Ylin = slab.sequential_dirk_linear(K, Md, A, tau, y0, Bst)
    Ynl, its = newton.sequential_dirk_newton(newton.LinearProblem(K, Md, b), A, c, tau, y0, G)
    np.testing.assert_allclose(Ynl, Ylin, rtol=1e-11, atol=1e-11)
    assert max(its) <= 2


def test_newton_quadratic_convergence_diffreact():
    dims = (8, 8, 1)
    prob = newton.DiffReactProblem(dims)
    tau = 0.05
    y0 = np.full(64, 0.5) + 0.3 * np.sin(np.arange(64))
    known = prob.mass(y0) / tau
    t = tau
    y = y0.copy()
    res = []
    for _ in range(6):
        G = prob.mass(y) / tau + prob.f(t, y) - known
        res.append(np.linalg.norm(G))
        J = sp.diags(prob.dmass(y) / tau) + prob.jac(t, y)
        y = y - sp.linalg.spsolve(J.tocsc(), G)
    # quadratic: e_{k+1} <= C e_k^2 with one C over three steps
    ratios = [res[k + 1] / res[k] ** 2 for k in (1, 2, 3)]
    assert max(ratios) < 1e-3 and res[4] < 1e-12 * res[0]


def _ode_order(tab, nsteps_list):
    """y' = -y + sin t, y(0)=1 as a 1x1 system; return errors at T = 1."""
    K = sp.csr_matrix(np.array([[1.0]]))
    Md = np.array([1.0])
    b = lambda t: np.array([math.sin(t)])
    exact = lambda t: 1.5 * math.exp(-t) + 0.5 * (math.sin(t) - math.cos(t))
    A, _, c = tab
    m = A.shape[0]
    errs = []
    for ns in nsteps_list:
        tau = 1.0 / ns
        Y, _ = newton.sequential_dirk_newton(newton.LinearProblem(K, Md, b), A, c, tau,
                                             np.array([1.0]), ns * m)
        errs.append(abs(Y[0, -1] - exact(1.0)))
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


def test_time_orders():
    r1 = _ode_order(coupling.implicit_euler(), [20, 40, 80])
    r2 = _ode_order(coupling.sdirk2(), [20, 40, 80])
    assert np.all(np.abs(r1 - 1.0) < 0.1), r1
    assert np.all(np.abs(r2 - 2.0) < 0.15), r2


def test_pipelined_linear_equals_sequential():
    K, Md, b, rng = _linear(5, 3)
    A, _, c = coupling.sdirk2()
    tau, G, s = 0.05, 6, 3
    y0 = rng.standard_normal(K.shape[0])
    prob = newton.LinearProblem(K, Md, b)
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, tau, y0, G)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, tau, y0, G, s, tol=1e-12,
                                            inner_tol=1e-6, precond="ilu0")
    np.testing.assert_allclose(Ypl, Yseq, rtol=1e-9, atol=1e-10)


def test_pipelined_diffreact_equals_sequential():
    dims = (8, 8, 1)
    prob = newton.DiffReactProblem(dims)
    A, _, c = coupling.sdirk2()
    tau, G = 0.01, 6
    y0 = np.full(64, 0.5)
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, tau, y0, G)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, tau, y0, G, 2, tol=1e-12,
                                            inner_tol=1e-6)
    np.testing.assert_allclose(Ypl, Yseq, rtol=1e-10, atol=1e-11)


def test_pipelined_richards_step_bound_8cube():
    """On 8^3 cells the trailing window columns' chord steps diverge without a
    step bound (the oracle reaches |psi| ~ 1e18); with max_step = 1 every
    window converges and the result equals sequential Newton stepping."""
    import synth
    dims = (8, 8, 8)
    Ks = np.exp(2.0 * synth.correlated_field(4, dims[::-1], 2.0))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    prob = newton.RichardsProblem(dims, Ks, vg, 1 / 16)
    A, _, c = coupling.implicit_euler()
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, 1 / 96, -z, 6)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, 1 / 96, -z, 6, 4, tol=1e-12,
                                            inner_tol=1e-6, max_newton=40, max_step=1.0)
    assert max(st["newton"]) < 40
    np.testing.assert_allclose(Ypl, Yseq, rtol=1e-9, atol=1e-10)


def test_pipelined_richards_equals_sequential():
    dims = (4, 4, 4)
    rng = np.random.default_rng(4)
    Ks = np.exp(rng.standard_normal(dims[::-1]))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    prob = newton.RichardsProblem(dims, Ks, vg, 1 / 16)
    A, _, c = coupling.implicit_euler()
    tau, G = 1 / 96, 5
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, tau, -z, G)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, tau, -z, G, 4, tol=1e-12,
                                            inner_tol=1e-6)
    np.testing.assert_allclose(Ypl, Yseq, rtol=1e-9, atol=1e-10)


def test_pipelined_richards_lscheme_equals_sequential():
    """Algorithm 1 with the L-scheme of Sec. 4.3 as the outer iteration (L =
    Lipschitz constant of theta, conductivities frozen at the first column)
    converges, linearly, to the same stages as sequential Newton stepping.
    The trailing columns iterate with the first column's frozen conductivities
    and need the step bound, as with Newton."""
    import synth
    dims = (6, 6, 6)
    Ks = np.exp(2.0 * synth.correlated_field(4, dims[::-1], 2.0))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    prob = newton.RichardsProblem(dims, Ks, vg, 1 / 16)
    A, _, c = coupling.implicit_euler()
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, 1 / 96, -z, 5)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, 1 / 96, -z, 5, 4, tol=1e-10,
                                            inner_tol=1e-8, max_newton=120, max_step=1.0,
                                            lscheme_L=vg.lipschitz())
    assert max(st["newton"]) < 120
    # ||R_0|| <= 1e-10 ||B0_0|| ~ 4e-8 and ||J^-1|| <= 1 here (diag J >= alpha
    # theta' >= 1 on these heads): stage errors below 1e-7
    np.testing.assert_allclose(Ypl, Yseq, rtol=0, atol=1e-7)


def test_pipelined_with_block_cg_and_bicgstab_equals_sequential():
    """Algorithm 1 with the paper's other block solvers as inner solves:
    block BiCGStab on the nonsymmetric diffusion-reaction Jacobian (the
    window's identical trailing columns are deflated at the start of each
    inner solve) and block CG on the symmetric positive definite L-scheme
    matrix of Richards' equation; both reach the stages of sequential Newton
    stepping."""
    import synth
    dims = (8, 8, 1)
    prob = newton.DiffReactProblem(dims)
    A, _, c = coupling.sdirk2()
    y0 = np.full(64, 0.5)
    Yseq, _ = newton.sequential_dirk_newton(prob, A, c, 0.01, y0, 6)
    Ypl, st = newton.pipelined_block_newton(prob, A, c, 0.01, y0, 6, 2, tol=1e-12,
                                            inner_tol=1e-6, solver="bicgstab")
    assert st["inner"] > 0
    np.testing.assert_allclose(Ypl, Yseq, rtol=1e-10, atol=1e-11)

    dims = (6, 6, 6)
    Ks = np.exp(2.0 * synth.correlated_field(4, dims[::-1], 2.0))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    rprob = newton.RichardsProblem(dims, Ks, vg, 1 / 16)
    A, _, c = coupling.implicit_euler()
    Yseq, _ = newton.sequential_dirk_newton(rprob, A, c, 1 / 96, -z, 5)
    Ypl, st = newton.pipelined_block_newton(rprob, A, c, 1 / 96, -z, 5, 4, tol=1e-10,
                                            inner_tol=1e-8, max_newton=120, max_step=1.0,
                                            lscheme_L=vg.lipschitz(), solver="cg")
    assert max(st["newton"]) < 120
    np.testing.assert_allclose(Ypl, Yseq, rtol=0, atol=1e-7)
