"""Randomised property checks of the oracle (CPU; hypothesis where it is
installed): the identities its pins rest on hold over many shapes and seeds,
not only the hand-picked cases."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupling, fv, krylov, slab

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

SETTINGS = dict(max_examples=60, deadline=None, derandomize=True)


@settings(**SETTINGS)
@given(n=st.integers(3, 40), s=st.integers(1, 6), seed=st.integers(0, 2 ** 31 - 1),
       dup=st.booleans(), zero=st.booleans())
def test_cholqr2_factorises_and_deflates(n, s, seed, dup, zero):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((max(n, s), s))
    if dup and s > 1:
        W[:, -1] = 3.0 * W[:, 0]
    if zero and s > 2:
        W[:, 1] = 0.0
    Q, R = krylov.cholqr2(W)
    np.testing.assert_allclose(Q @ R, W, atol=1e-10 * max(1.0, np.abs(W).max()))
    live = np.abs(np.diag(R)) > 0
    np.testing.assert_allclose(Q[:, live].T @ Q[:, live], np.eye(live.sum()), atol=1e-12)
    assert np.all(Q[:, ~live] == 0.0)
    assert np.allclose(np.tril(R, -1), 0.0)


@settings(**SETTINGS)
@given(nx=st.integers(2, 6), ny=st.integers(1, 5), nz=st.integers(1, 4),
       seed=st.integers(0, 2 ** 31 - 1))
def test_stencil_ilu0_equals_generic_on_random_grids(nx, ny, nz, seed):
    dims = (nx, ny, nz)
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    v = tuple(rng.uniform(-2, 2, 3))
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), v)
    J = sp.csr_matrix(sp.diags(5.0 + rng.uniform(0, 1, n)) + K)
    J.sort_indices()
    L, U = krylov.ilu0(J)
    fac = krylov.ilu0_stencil(dims, J)
    X = rng.standard_normal((n, 2))
    np.testing.assert_allclose(krylov.ilu0_stencil_apply(dims, fac, X),
                               krylov.ilu0_apply(L, U)(X), rtol=1e-11, atol=1e-13)


@settings(**SETTINGS)
@given(s=st.integers(1, 5), seed=st.integers(0, 2 ** 31 - 1), lower=st.booleans())
def test_coupled_residual_is_the_kronecker_defect(s, seed, lower):
    """M Y A1^T + (K Y - B) A2^T - B0 equals (A1 (x) M + A2 (x) K) vec Y -
    (A2 (x) I) vec B - vec B0 with column-stacking vec, for any A1, A2."""
    rng = np.random.default_rng(seed)
    dims = (3, 2, 2)
    n = 12
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (1.0, 0.5, 0.0))
    M = rng.uniform(0.5, 2.0, n)
    A1, A2 = rng.standard_normal((s, s)), rng.standard_normal((s, s))
    if lower:
        A1, A2 = np.tril(A1), np.tril(A2)
    Y, B, B0 = (rng.standard_normal((n, s)) for _ in range(3))
    R = slab.coupled_residual(K, M, A1, A2, Y, B, B0)
    big = slab.kron_operator(K, M, A1, A2)
    vec = lambda Z: Z.reshape(-1, order="F")
    ref = big @ vec(Y) - np.kron(A2, np.eye(n)) @ vec(B) - vec(B0)
    np.testing.assert_allclose(vec(R), ref, rtol=1e-12, atol=1e-12)


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), s=st.integers(1, 5), vel=st.floats(0.0, 60.0))
def test_block_bicgstab_and_gmres_solve_random_nonsymmetric_blocks(seed, s, vel):
    rng = np.random.default_rng(seed)
    dims = (6, 5, 1)
    n = 30
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (vel, -vel / 2, 0.0))
    J = sp.csr_matrix(sp.identity(n) / 1e-2 + K)
    J.sort_indices()
    B = rng.standard_normal((n, s))
    Xd = np.linalg.solve(J.toarray(), B)
    L, U = krylov.ilu0(J)
    Pinv = krylov.ilu0_apply(L, U)
    for solve in (lambda: krylov.block_bicgstab(lambda V: J @ V, Pinv, B, 1e-12),
                  lambda: krylov.block_gmres(lambda V: J @ V, Pinv, B, 1e-12)):
        X, info = solve()
        assert info["converged"]
        np.testing.assert_allclose(X, Xd, rtol=1e-8, atol=1e-10)


@settings(**SETTINGS)
@given(s=st.integers(1, 6), seed=st.integers(0, 2 ** 31 - 1))
def test_slab_equals_sequential_stepping_for_random_slabs(s, seed):
    rng = np.random.default_rng(seed)
    dims = (5, 4, 2)
    n = 40
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (3.0, 1.0, 0.5))
    A, _, _ = coupling.implicit_euler()
    tau = 10.0 ** rng.uniform(-3, -1)
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    B = rng.uniform(-1, 1, (n, s))
    Y, info = slab.slab_solve(K, np.ones(n), A1, A2, B, tol=1e-12, inner_tol=1e-2,
                              precond="ilu0")
    Ys = slab.sequential_dirk_linear(K, np.ones(n), A, tau, np.zeros(n), B)
    assert info["converged"]
    np.testing.assert_allclose(Y, Ys, rtol=1e-9, atol=1e-12)


@settings(**SETTINGS)
@given(s=st.integers(1, 5), seed=st.integers(0, 2 ** 31 - 1), mgs=st.booleans(),
       pc=st.sampled_from(["none", "jacobi"]), nx=st.integers(2, 5), ny=st.integers(1, 4))
def test_global_gmres_reaches_the_dense_solution_with_either_orthogonalisation(
        s, seed, mgs, pc, nx, ny):
    """Global GMRES on the unsplit operator, with modified or two classical
    Gram-Schmidt passes, solves random small slabs (random log-normal
    diffusion, random velocity, theta-method coupling with its first stage
    eliminated, random B and B0) to the dense all-at-once solution."""
    rng = np.random.default_rng(seed)
    dims = (nx, ny, 2)
    n = nx * ny * 2
    D = np.exp(rng.standard_normal(n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, tuple(rng.uniform(0.0, 3.0, 3)))
    A, _, _ = coupling.theta_method(0.5)
    A1, A2, _ = coupling.multistep_matrices(A, s, 1e-2, eliminate_first=True)
    B = rng.standard_normal((n, s))
    B0 = rng.standard_normal((n, s))
    Y, info = slab.slab_solve_global(K, np.ones(n), A1, A2, B, B0, tol=1e-12, precond=pc,
                                     restart=8, ortho="mgs" if mgs else "cgs2")
    assert info["converged"]
    Yd = slab.solve_all_at_once_dense(K, np.ones(n), A1, A2, B, B0)
    err = np.linalg.norm(Y - Yd, axis=0) / np.linalg.norm(Yd, axis=0)
    assert np.all(err < 1e-9), err
