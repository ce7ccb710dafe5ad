"""Pins of oracle.krylov: CholQR2, minimal-residual property of block GMRES,
exact termination, ILU(0) definition (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fv, krylov


def _J(n=6, seed=0, d3=False, tau=0.01):
    dims = (n, n, n) if d3 else (n, n, 1)
    rng = np.random.default_rng(seed)
    D = np.exp(rng.standard_normal(dims[::-1]))
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    N = int(np.prod(dims))
    J = sp.csr_matrix(sp.identity(N) / tau + K)
    J.sort_indices()
    return J, rng


def test_cholqr2_orthonormal_and_factor():
    rng = np.random.default_rng(1)
    W = rng.standard_normal((200, 6)) @ np.diag([1, 1e-3, 1, 1e3, 1, 1])
    Q, R = krylov.cholqr2(W)
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-13)
    np.testing.assert_allclose(Q @ R, W, rtol=1e-12, atol=1e-10)
    assert np.allclose(np.tril(R, -1), 0.0)


def test_cholqr_deflates_dependent_columns():
    rng = np.random.default_rng(2)
    W = rng.standard_normal((100, 4))
    W[:, 2] = W[:, 0]                 # duplicate column
    W[:, 3] = 0.0                     # zero column
    Q, R = krylov.cholqr2(W)
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(R))
    np.testing.assert_allclose(Q[:, 2], 0.0)
    np.testing.assert_allclose(Q[:, 3], 0.0)
    np.testing.assert_allclose(Q @ R, W, atol=1e-12)
    np.testing.assert_allclose(Q[:, :2].T @ Q[:, :2], np.eye(2), atol=1e-13)


def _krylov_min_residual(J, R, k):
    """Per-column minimum of ||R_i - J Z c|| over the block Krylov space
    span{R, J R, ..., J^{k-1} R} (explicit basis + least squares)."""
    blocks = [R]
    for _ in range(k - 1):
        blocks.append(J @ blocks[-1])
    Z = np.hstack(blocks)
    Zq, _ = np.linalg.qr(Z)
    JZ = J @ Zq
    res = []
    for i in range(R.shape[1]):
        c, *_ = np.linalg.lstsq(JZ, R[:, i], rcond=None)
        res.append(np.linalg.norm(R[:, i] - JZ @ c))
    return np.array(res)


@pytest.mark.parametrize("s", [1, 3])
def test_block_gmres_minimal_residual_property(s):
    """After k block steps (no restart, no preconditioner) each column's residual
    is the minimum over the block Krylov space: the defining property of
    (block) GMRES; for s = 1 this is textbook GMRES."""
    J, rng = _J(5, 3)
    R = rng.standard_normal((J.shape[0], s))
    ident = lambda X: X.copy()
    for k in (1, 2, 4):
        X, info = krylov.block_gmres(lambda X: J @ X, ident, R, tol=0.0, restart=30, maxit=k)
        true = np.linalg.norm(R - J @ X, axis=0)
        best = _krylov_min_residual(J, R, k)
        np.testing.assert_allclose(true, best, rtol=1e-7, atol=1e-10)
        np.testing.assert_allclose(info["est"], true, rtol=1e-7, atol=1e-10)


def test_block_gmres_exact_termination_and_diagonal():
    J, rng = _J(3, 4)                   # N = 9
    N = J.shape[0]
    R = rng.standard_normal((N, 3))
    X, info = krylov.block_gmres(lambda X: J @ X, lambda X: X.copy(), R, tol=1e-12,
                                 restart=30)
    assert info["converged"] and info["iters"] <= 3
    np.testing.assert_allclose(J @ X, R, rtol=1e-9, atol=1e-9)
    D = sp.diags(rng.uniform(1, 10, 50)).tocsr()
    R = rng.standard_normal((50, 4))
    X, info = krylov.block_gmres(lambda X: D @ X, krylov.jacobi(D), R, tol=1e-12)
    assert info["iters"] == 1
    np.testing.assert_allclose(D @ X, R, rtol=1e-12)


def test_block_gmres_restarted_preconditioned():
    J, rng = _J(6, 5, d3=True)
    R = rng.uniform(-1, 1, (J.shape[0], 4))
    for kind in ("jacobi", "ilu0"):
        X, info = krylov.block_gmres(lambda X: J @ X, krylov.make_preconditioner(J, kind),
                                     R, tol=1e-10, restart=5)
        assert info["converged"]
        rel = np.linalg.norm(R - J @ X, axis=0) / np.linalg.norm(R, axis=0)
        assert np.all(rel < 2e-10)


def test_block_gmres_zero_and_duplicate_columns():
    J, rng = _J(5, 6)
    R = rng.standard_normal((J.shape[0], 4))
    R[:, 1] = 0.0
    R[:, 3] = 2.0 * R[:, 0]
    X, info = krylov.block_gmres(lambda X: J @ X, krylov.jacobi(J), R, tol=1e-10)
    assert info["converged"] and np.all(np.isfinite(X))
    np.testing.assert_allclose(X[:, 1], 0.0)
    np.testing.assert_allclose(X[:, 3], 2.0 * X[:, 0], rtol=1e-8, atol=1e-12)


def test_ilu0_tridiagonal_is_exact_lu():
    n = 30
    rng = np.random.default_rng(7)
    T = sp.diags([rng.uniform(-1, 0, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, 0, n - 1)],
                 [-1, 0, 1], format="csr")
    L, U = krylov.ilu0(T)
    np.testing.assert_allclose((L @ U).toarray(), T.toarray(), atol=1e-13)
    b = rng.standard_normal((n, 2))
    np.testing.assert_allclose(T @ krylov.ilu0_apply(L, U)(b), b, atol=1e-12)


def _dense_ilu0(A):
    """Brute force ILU(0) on a dense copy with the sparsity mask (IKJ)."""
    A = A.copy()
    n = A.shape[0]
    mask = A != 0
    for i in range(1, n):
        for k in range(i):
            if not mask[i, k]:
                continue
            A[i, k] /= A[k, k]
            for j in range(k + 1, n):
                if mask[i, j]:
                    A[i, j] -= A[i, k] * A[k, j]
    return np.tril(A, -1) + np.eye(n), np.triu(A)


def test_ilu0_matches_brute_force_and_pattern_property():
    J, _ = _J(5, 8, d3=True)
    L, U = krylov.ilu0(J)
    Ld, Ud = _dense_ilu0(J.toarray())
    np.testing.assert_allclose(L.toarray(), Ld, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(U.toarray(), Ud, rtol=1e-12, atol=1e-12)
    # defining property of ILU(0): (L U)_ij = a_ij on the pattern of A
    LU = (L @ U).toarray()
    Jd = J.toarray()
    mask = Jd != 0
    np.testing.assert_allclose(LU[mask], Jd[mask], rtol=1e-12, atol=1e-9)
    assert L.nnz + U.nnz == J.nnz + J.shape[0]


@pytest.mark.parametrize("dims", [(5, 4, 3), (7, 6, 1), (2, 3, 4), (1, 5, 2), (3, 1, 4),
                                  (9, 1, 1)])
def test_ilu0_stencil_equals_generic_ilu0(dims):
    """The plane-by-plane stencil ILU(0) gives the same factors and the same
    P^{-1} X as the generic IKJ elimination, including grids with axes of
    extent 1 (where stencil offsets coincide)."""
    n = int(np.prod(dims))
    rng = np.random.default_rng(11)
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (1.0, -0.5, 0.3))
    J = sp.csr_matrix(sp.diags(10.0 + rng.uniform(-1, 1, n)) + K)
    J.sort_indices()
    L, U = krylov.ilu0(J)
    d, lower, upper = krylov.ilu0_stencil(dims, J)
    np.testing.assert_allclose(d, U.diagonal(), rtol=1e-13)
    Uoff = sp.triu(U, k=1).toarray()
    for o, u in upper.items():
        idx = np.nonzero(u)[0]
        np.testing.assert_array_equal(Uoff[idx, idx + o], u[idx])   # U keeps J's upper part
    X = rng.standard_normal((n, 3))
    np.testing.assert_allclose(krylov.ilu0_stencil_apply(dims, (d, lower, upper), X),
                               krylov.ilu0_apply(L, U)(X), rtol=1e-12, atol=1e-13)


def test_ilu0_stencil_tridiagonal_is_exact_solve():
    """On a 1-D grid ILU(0) is the exact LU: P^{-1} = J^{-1}."""
    dims = (40, 1, 1)
    rng = np.random.default_rng(12)
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal((1, 1, 40))), (1.0, 0.0, 0.0))
    J = sp.csr_matrix(sp.identity(40) * 50.0 + K)
    b = rng.standard_normal((40, 2))
    Z = krylov.ilu0_stencil_apply(dims, krylov.ilu0_stencil(dims, J), b)
    np.testing.assert_allclose(J @ Z, b, rtol=1e-12, atol=1e-12)


def _spd(n=7, seed=5):
    """SPD 5-point diffusion matrix plus a mass term on an n x n grid."""
    dims = (n, n, 1)
    rng = np.random.default_rng(seed)
    K = fv.convdiff_matrix(dims, np.exp(rng.standard_normal(dims[::-1])), (0.0, 0.0, 0.0))
    J = sp.csr_matrix(K + 50.0 * sp.identity(n * n))
    J.sort_indices()
    return J, rng


def test_block_cg_single_column_is_textbook_pcg():
    J, rng = _spd()
    b = rng.standard_normal((J.shape[0], 1))
    d = J.diagonal()
    X, info = krylov.block_cg(lambda V: J @ V, lambda V: V / d[:, None], b, 1e-12)
    # textbook PCG, written out
    x = np.zeros_like(b[:, 0]); r = b[:, 0].copy(); z = r / d; p = z.copy(); it = 0
    while np.linalg.norm(r) > 1e-12 * np.linalg.norm(b):
        q = J @ p; al = (r @ z) / (p @ q); x += al * p; rn = r - al * q
        zn = rn / d; be = (rn @ zn) / (r @ z); p = zn + be * p; r, z = rn, zn; it += 1
    assert info["converged"] and abs(info["iters"] - it) <= 1
    np.testing.assert_allclose(X[:, 0], x, rtol=1e-9, atol=1e-12)


def test_block_cg_solves_spd_blocks_and_survives_dependent_columns():
    J, rng = _spd(9, 6)
    n = J.shape[0]
    B = rng.standard_normal((n, 5))
    B[:, 3] = 2.0 * B[:, 0]                       # dependent column: rank 4
    B[:, 4] = 0.0                                 # zero column
    L, U = krylov.ilu0(J)
    Minv = krylov.ilu0_apply(L, U)
    X, info = krylov.block_cg(lambda V: J @ V, Minv, B, 1e-11)
    assert info["converged"] and np.all(np.isfinite(X))
    Xd = np.linalg.solve(J.toarray(), B)
    np.testing.assert_allclose(X, Xd, rtol=1e-8, atol=1e-12)
    # the block needs no more iterations than its hardest single column
    its1 = max(krylov.block_cg(lambda V: J @ V, Minv, B[:, [k]], 1e-11)[1]["iters"]
               for k in range(3))
    assert info["iters"] <= its1


def _nonsym(n=9, seed=8, vel=(40.0, 20.0, 0.0)):
    """Nonsymmetric convection-diffusion matrix (upwind, strong convection)
    plus a mass term on an n x (n-1) grid."""
    dims = (n, n - 1, 1)
    rng = np.random.default_rng(seed)
    K = fv.convdiff_matrix(dims, np.exp(0.5 * rng.standard_normal(dims[::-1])), vel)
    J = sp.csr_matrix(sp.identity(K.shape[0]) / 1e-2 + K)
    J.sort_indices()
    return J, rng


def test_block_bicgstab_single_column_is_library_bicgstab():
    """s = 1 reduces to textbook BiCGStab: the iterates after k = 1, 2, 3, 6
    steps equal scipy's right-preconditioned BiCGStab (an independent
    implementation) to rounding."""
    from scipy.sparse.linalg import LinearOperator, bicgstab
    J, rng = _nonsym()
    b = rng.standard_normal((J.shape[0], 1))
    L, U = krylov.ilu0(J)
    Minv = krylov.ilu0_apply(L, U)
    M = LinearOperator(J.shape, matvec=lambda v: Minv(v.reshape(-1, 1)).ravel())
    for k in (1, 2, 3, 6):
        X, info = krylov.block_bicgstab(lambda V: J @ V, Minv, b, 1e-30, maxit=k)
        x, _ = bicgstab(J, b[:, 0], rtol=1e-30, atol=0.0, maxiter=k, M=M)
        assert info["iters"] == k
        np.testing.assert_allclose(X[:, 0], x, rtol=1e-11, atol=1e-13 * np.abs(x).max())


def test_block_bicgstab_coefficients_satisfy_their_defining_equations():
    """alpha makes S orthogonal to the shadow block (Rt^T S = 0), omega
    minimises ||S - omega T||_F (<T, Rh>_F = 0) and beta makes
    Rt^T (T + V beta) = 0: each fails for a transposed s x s solve or a
    flipped sign."""
    J, rng = _nonsym(10, 9)
    B = rng.standard_normal((J.shape[0], 4))
    rec = []
    krylov.block_bicgstab(lambda V: J @ V, lambda V: V / J.diagonal()[:, None], B, 1e-10,
                          record=rec)
    assert len(rec) >= 3
    for r in rec:
        assert np.abs(r["RtS"]).max() <= 1e-10
        assert abs(r["omega_orth"]) <= 1e-10
        if "RtTVb" in r:
            assert np.abs(r["RtTVb"]).max() <= 1e-10


def test_block_bicgstab_solves_and_survives_dependent_columns():
    J, rng = _nonsym(9, 10)
    n = J.shape[0]
    B = rng.standard_normal((n, 6))
    B[:, 3] = -3.0 * B[:, 1]                      # dependent column
    B[:, 4] = 0.0                                 # zero column
    B[:, 5] = B[:, 0]                             # duplicate column
    L, U = krylov.ilu0(J)
    X, info = krylov.block_bicgstab(lambda V: J @ V, krylov.ilu0_apply(L, U), B, 1e-11)
    assert info["converged"] and np.all(np.isfinite(X))
    Xd = np.linalg.solve(J.toarray(), B)
    np.testing.assert_allclose(X, Xd, rtol=1e-8, atol=1e-12)
    np.testing.assert_array_equal(X[:, 4], 0.0)
    np.testing.assert_allclose(X[:, 5], X[:, 0], rtol=1e-12, atol=1e-15)


def test_block_gmres_never_worse_than_its_columns_alone():
    """The block Krylov space of k steps contains every column's own Krylov
    space of k steps, so after k block steps each column's residual is at
    most that of GMRES run on the column alone (the motivation of block
    Krylov methods, Sec. 1); with right preconditioning the same holds for
    the preconditioned spaces."""
    J, rng = _J(6, 12)
    R = rng.standard_normal((J.shape[0], 4))
    ilu = krylov.make_preconditioner(J, "ilu0")
    for P in (lambda X: X.copy(), ilu):
        for k in (1, 3, 6):
            X, _ = krylov.block_gmres(lambda X: J @ X, P, R, tol=0.0, restart=30, maxit=k)
            blk = np.linalg.norm(R - J @ X, axis=0)
            for i in range(R.shape[1]):
                x1, _ = krylov.block_gmres(lambda X: J @ X, P, R[:, [i]], tol=0.0, restart=30,
                                           maxit=k)
                one = np.linalg.norm(R[:, i] - J @ x1[:, 0])
                assert blk[i] <= one * (1.0 + 1e-9) + 1e-13
