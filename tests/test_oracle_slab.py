"""Pins of oracle.slab: Kronecker identity, all-at-once == sequential
stepping, nilpotent splitting, slab solve to tolerance (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupling, fv, krylov, slab


def _problem(n=5, seed=0, v=(1.0, 0.5, 0.0), d3=False):
    dims = (n, n, n) if d3 else (n, n, 1)
    rng = np.random.default_rng(seed)
    D = np.exp(rng.standard_normal(dims[::-1]))
    K = fv.convdiff_matrix(dims, D, v)
    Md = 1.0 + 0.5 * rng.random(int(np.prod(dims)))
    return K, Md, rng


def test_kronecker_vec_identity():
    """(C (x) M) vec(Y) = vec(M Y C^T) for the column-stacking vec."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((5, 5))
    C = rng.standard_normal((3, 3))
    Y = rng.standard_normal((5, 3))
    lhs = np.kron(C, M) @ slab.vec(Y)
    rhs = slab.vec(M @ Y @ C.T)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)
    # and the block-diagonal statement of Sec. 2.1: (I (x) A) vec(X) = vec(A X)
    np.testing.assert_allclose(np.kron(np.eye(3), M) @ slab.vec(Y), slab.vec(M @ Y), atol=1e-13)


def test_coupled_residual_is_kronecker_defect():
    K, Md, rng = _problem(4, 1)
    n = K.shape[0]
    s = 3
    A1 = rng.standard_normal((s, s))
    A2 = rng.standard_normal((s, s))
    Y, B, B0 = rng.standard_normal((3, n, s))
    R = slab.coupled_residual(K, Md, A1, A2, Y, B, B0)
    Kr = slab.kron_operator(K, Md, A1, A2)
    rhs = np.kron(A2, np.eye(n)) @ slab.vec(B) + slab.vec(B0)
    np.testing.assert_allclose(slab.vec(R), Kr @ slab.vec(Y) - rhs, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("tab,steps", [("ie", 4), ("sdirk2", 3), ("theta", 3)])
def test_all_at_once_equals_sequential(tab, steps):
    """Stiffly accurate: the s-step all-at-once solve equals s sequential steps
    (Eq. time-stepping-matrices-multiple-parallel-time-steps and the identity
    y^{n+i} = y^{(n+i-1,m)})."""
    K, Md, rng = _problem(4, 2)
    n = K.shape[0]
    tau = 0.05
    y0 = rng.standard_normal(n)
    if tab == "ie":
        A, b, c = coupling.implicit_euler()
    elif tab == "sdirk2":
        A, b, c = coupling.sdirk2()
    else:
        A, b, c = coupling.theta_method(0.5)
    m = A.shape[0]
    Bst = rng.standard_normal((n, steps * m))
    if tab == "theta":            # b(t^{n+1}) is shared by stages (n,2) and (n+1,1)
        for k in range(1, steps):
            Bst[:, 2 * k] = Bst[:, 2 * k - 1]
    Yseq = slab.sequential_dirk_linear(K, Md, A, tau, y0, Bst)
    if tab == "theta":
        A1, A2, e = coupling.multistep_matrices(A, steps, tau, eliminate_first=True)
        B = Bst[:, 1::2]
        B0 = np.zeros((n, steps))
        B0[:, 0] = Md * y0 / tau + e[0] * (Bst[:, 0] - K @ y0)
        Y = slab.solve_all_at_once_dense(K, Md, A1, A2, B, B0)
        np.testing.assert_allclose(Y, Yseq[:, 1::2], rtol=1e-10, atol=1e-11)
    else:
        A1, A2, _ = coupling.multistep_matrices(A, steps, tau)
        B0 = np.zeros((n, steps * m))
        B0[:, :m] = (Md * y0 / tau)[:, None]
        Y = slab.solve_all_at_once_dense(K, Md, A1, A2, Bst, B0)
        np.testing.assert_allclose(Y, Yseq, rtol=1e-10, atol=1e-11)


def test_fixed_point_exact_after_s_iterations():
    """With exact inner solves the split-off parts are strictly lower
    triangular, so column k is exact after k+1 outer iterations and the whole
    slab after s (derived from Eq. matrix-fixed-point-equation)."""
    K, Md, rng = _problem(5, 4)
    n = K.shape[0]
    s, tau = 5, 0.02
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    B = rng.standard_normal((n, s))
    y0 = rng.standard_normal(n)
    B0 = np.zeros((n, s))
    B0[:, 0] = Md * y0 / tau
    Yex = slab.solve_all_at_once_dense(K, Md, A1, A2, B, B0)
    for outer in range(1, s + 1):
        Y, info = slab.slab_solve(K, Md, A1, A2, B, B0, tol=0.0, exact_inner=True,
                                  max_outer=outer)
        err = np.linalg.norm(Y - Yex, axis=0) / np.linalg.norm(Yex, axis=0)
        assert np.all(err[:outer] < 1e-12)
        if outer < s:
            assert err[outer] > 1e-6
    # s = 1 needs exactly one outer iteration (Sec. 4.1 remark on s = 1)
    A1b, A2b, _ = coupling.multistep_matrices(A, 1, tau)
    Y1, info = slab.slab_solve(K, Md, A1b, A2b, B[:, :1], B0[:, :1], tol=1e-12,
                               exact_inner=True)
    assert info["outer"] == 1


@pytest.mark.parametrize("precond", ["jacobi", "ilu0"])
def test_slab_solve_block_gmres_reaches_tolerance(precond):
    K, Md, rng = _problem(6, 5, d3=True)
    n = K.shape[0]
    s, tau = 4, 1e-2
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    B = rng.uniform(-1, 1, (n, s))
    Y, info = slab.slab_solve(K, Md, A1, A2, B, None, tol=1e-12, inner_tol=1e-2,
                              precond=precond, restart=10)
    assert info["converged"]
    Yex = slab.sequential_dirk_linear(K, Md, A, tau, np.zeros(n), B)
    err = np.linalg.norm(Y - Yex, axis=0) / np.linalg.norm(Yex, axis=0)
    assert np.all(err < 1e-9)


def test_planted_transpose_in_coupling_is_caught(monkeypatch):
    """A plausible mistake (A2 used without transpose in the residual) breaks
    the all-at-once == sequential pin."""
    orig = slab.coupled_residual

    def wrong(K, Mdiag, A1, A2, Y, B=None, B0=None):
        return orig(K, Mdiag, A1.T, A2.T, Y, B, B0)

    K, Md, rng = _problem(4, 6)
    n = K.shape[0]
    s, tau = 3, 0.05
    A, _, _ = coupling.sdirk2()
    A1, A2, _ = coupling.multistep_matrices(A, 2, tau)
    y0 = rng.standard_normal(n)
    Bst = rng.standard_normal((n, 4))
    B0 = np.zeros((n, 4))
    B0[:, :2] = (Md * y0 / tau)[:, None]
    Yseq = slab.sequential_dirk_linear(K, Md, A, tau, y0, Bst)
    monkeypatch.setattr(slab, "coupled_residual", wrong)
    Y, info = slab.slab_solve(K, Md, A1, A2, Bst, B0, tol=1e-12, exact_inner=True,
                              max_outer=30)
    assert not np.allclose(Y, Yseq, rtol=1e-6)


def test_narrowed_inner_solves_keep_the_solution_and_iterations():
    """Leaving converged leading columns out of the inner solve (lower
    triangular coupling) reaches the same slab solution with fewer
    column-steps (Arnoldi steps times block width), at most one more outer
    iteration, and every column meets the tolerance."""
    rng = np.random.default_rng(21)
    dims = (10, 9, 1)
    n, s = 90, 8
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (1.0, 0.5, 0.0))
    tau = 1e-2
    A1 = (np.eye(s) - np.eye(s, k=-1)) / tau
    A2 = np.eye(s)
    B = rng.uniform(-1, 1, (n, s))
    Y0, i0 = slab.slab_solve(K, np.ones(n), A1, A2, B, tol=1e-12, inner_tol=1e-2,
                             precond="ilu0")
    Y1, i1 = slab.slab_solve(K, np.ones(n), A1, A2, B, tol=1e-12, inner_tol=1e-2,
                             precond="ilu0", narrow=True)
    assert i0["converged"] and i1["converged"]
    assert i1["outer"] <= i0["outer"] + 1
    assert i1["column_steps"] < i0["column_steps"]
    np.testing.assert_allclose(Y1, Y0, rtol=0, atol=1e-9 * np.abs(Y0).max())
    R = slab.coupled_residual(K, np.ones(n), A1, A2, Y1, B)
    F = slab.rhs_F(A2, B)
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-12 * np.linalg.norm(F, axis=0))


def test_slab_with_block_cg_equals_sequential_stepping():
    """Pure diffusion (symmetric J): the slab solved with block CG inner
    solves equals s sequential implicit-Euler steps."""
    rng = np.random.default_rng(23)
    dims = (8, 7, 3)
    n, s, tau = 168, 4, 1e-2
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (0.0, 0.0, 0.0))
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    B = rng.uniform(-1, 1, (n, s))
    Y, info = slab.slab_solve(K, np.ones(n), A1, A2, B, tol=1e-12, inner_tol=1e-2,
                              precond="ilu0", solver="cg")
    Ys = slab.sequential_dirk_linear(K, np.ones(n), A, tau, np.zeros(n), B)
    assert info["converged"] and info["inner"] > 0
    np.testing.assert_allclose(Y, Ys, rtol=1e-9, atol=1e-12)


def test_slab_with_block_bicgstab_equals_sequential_stepping():
    """Convection-diffusion (nonsymmetric J): the slab solved with block
    BiCGStab inner solves (Sec. 4.1's solver for this problem) equals s
    sequential implicit-Euler steps, with and without narrowed inner solves."""
    rng = np.random.default_rng(29)
    dims = (8, 7, 3)
    n, s, tau = 168, 4, 1e-2
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (30.0, 15.0, 5.0))
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    B = rng.uniform(-1, 1, (n, s))
    Ys = slab.sequential_dirk_linear(K, np.ones(n), A, tau, np.zeros(n), B)
    for pc in ("ilu0", "jacobi"):
        for narrow in (False, True):
            Y, info = slab.slab_solve(K, np.ones(n), A1, A2, B, tol=1e-12, inner_tol=1e-2,
                                      precond=pc, solver="bicgstab", narrow=narrow)
            assert info["converged"] and info["inner"] > 0
            np.testing.assert_allclose(Y, Ys, rtol=1e-9, atol=1e-12)


def test_sequential_stepping_iterative_stage_solves_equal_lu():
    """The GMRES option of sequential_dirk_linear (for grids where sparse LU
    is too slow) gives the LU result: 3-D convection-diffusion with a
    log-normal coefficient, 12^3 cells, 6 implicit-Euler steps and 3 steps of
    the theta example (explicit first stage)."""
    import synth
    dims = (12, 12, 12)
    n = 12 ** 3
    D = np.exp(synth.normal(5, n)).reshape(12, 12, 12)
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    B = synth.uniform(6, n * 6).reshape(n, 6)
    y0 = synth.uniform(7, n)
    for A in (coupling.implicit_euler()[0], coupling.theta_method(0.5)[0]):
        lu = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, y0, B)
        it = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, y0, B, rtol=1e-15)
        rel = np.linalg.norm(it - lu, axis=0) / np.linalg.norm(lu, axis=0)
        assert np.all(rel < 1e-12), rel


def _small_slab(s=4, dims=(9, 8, 1), seed=3):
    import synth
    n = int(np.prod(dims))
    D = np.exp(synth.normal(seed, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, 1e-3)
    B = synth.uniform(seed + 1, n * s).reshape(n, s)
    return K, n, A, A1, A2, B


@pytest.mark.parametrize("ortho", ["cgs2", "mgs"])
@pytest.mark.parametrize("precond", ["none", "jacobi", "ilu0"])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_global_gmres_cycle_is_the_minimum_residual_over_its_krylov_space(precond, k, ortho):
    """One cycle of k steps of global GMRES from Y = 0: the residual's
    Frobenius norm equals min over Z in span{R, A P R, ..., (A P)^(k-1) R} of
    ||R - A P Z||_F, computed here by a dense least squares on the vec'd
    Krylov matrices (the defining property of GMRES in the Frobenius inner
    product, independent of how the iteration gets there)."""
    K, n, A, A1, A2, B = _small_slab()
    Y, info = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-300, precond=precond,
                                     restart=k, max_outer=1, ortho=ortho)
    assert info["cycles"] == 1 and info["inner"] == k
    R1 = slab.coupled_residual(K, np.ones(n), A1, A2, Y, B)
    alpha, beta = A1[0, 0], A2[0, 0]
    J = sp.csr_matrix(sp.identity(n) * alpha + beta * K)
    P = krylov.make_preconditioner(J, precond)
    Aop = lambda V: slab.coupled_residual(K, np.ones(n), A1, A2, V)
    R0 = slab.coupled_residual(K, np.ones(n), A1, A2, np.zeros_like(B), B)
    # an orthonormal basis of the Krylov space (each new direction A P q of
    # the last basis vector, orthonormalised by numpy's QR), well conditioned
    # unlike the power basis
    Q = slab.vec(R0)[:, None] / np.linalg.norm(R0)
    while Q.shape[1] < k:
        v = slab.vec(Aop(P(slab.unvec(Q[:, -1], n, A1.shape[0]))))
        Q = np.linalg.qr(np.column_stack([Q, v]))[0]
    Mk = np.column_stack([slab.vec(Aop(P(slab.unvec(q, n, A1.shape[0])))) for q in Q.T])
    c, *_ = np.linalg.lstsq(Mk, slab.vec(R0), rcond=None)
    best = np.linalg.norm(slab.vec(R0) - Mk @ c)
    assert np.linalg.norm(R1) == pytest.approx(best, rel=1e-7, abs=1e-12 * np.linalg.norm(R0))


@pytest.mark.parametrize("ortho", ["cgs2", "mgs"])
@pytest.mark.parametrize("precond", ["jacobi", "ilu0"])
def test_global_gmres_slab_equals_sequential_stepping(precond, ortho):
    K, n, A, A1, A2, B = _small_slab(s=5, dims=(7, 6, 5))
    Y, info = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-13, precond=precond,
                                     restart=10, ortho=ortho)
    assert info["converged"]
    Yseq = slab.sequential_dirk_linear(K, np.ones(n), A, 1e-3, np.zeros(n), B)
    Yd = slab.solve_all_at_once_dense(K, np.ones(n), A1, A2, B)
    for ref in (Yseq, Yd):
        err = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.all(err < 1e-11), err


def test_global_gmres_mgs_basis_is_orthonormal_and_satisfies_the_arnoldi_relation():
    """Modified Gram-Schmidt in the Frobenius inner product: the Krylov basis
    is orthonormal to rounding level on this well-conditioned slab and the
    Arnoldi relation A P V_k = V_{k+1} H_k holds; the MGS solver meets tol
    within one step per restart of the CGS2 one."""
    K, n, A, A1, A2, B = _small_slab(s=4, dims=(9, 8, 3))
    alpha, beta = A1[0, 0], A2[0, 0]
    J = sp.csr_matrix(sp.identity(n) * alpha + beta * K)
    P = krylov.make_preconditioner(J, "jacobi")
    Aop = lambda V: slab.coupled_residual(K, np.ones(n), A1, A2, P(V))
    R0 = slab.coupled_residual(K, np.ones(n), A1, A2, np.zeros_like(B), B)
    k = 12
    V = [R0 / np.sqrt(np.sum(R0 * R0))]
    H = np.zeros((k + 1, k))
    for j in range(k):                  # the Arnoldi process with MGS, by hand
        W = Aop(V[j])
        for i in range(j + 1):
            H[i, j] = np.sum(V[i] * W)
            W = W - H[i, j] * V[i]
        H[j + 1, j] = np.sqrt(np.sum(W * W))
        V.append(W / H[j + 1, j])
    G = np.array([[np.sum(a * b) for b in V] for a in V])
    assert np.max(np.abs(G - np.eye(k + 1))) < 1e-10
    lhs = np.column_stack([slab.vec(Aop(V[j])) for j in range(k)])
    rhs = np.column_stack([slab.vec(v) for v in V]) @ H
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(lhs)
    _, ia = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-10, restart=30)
    Ym, im = slab.slab_solve_global(K, np.ones(n), A1, A2, B, tol=1e-10, restart=30,
                                    ortho="mgs")
    assert im["converged"] and abs(im["inner"] - ia["inner"]) <= 1 + ia["cycles"]
