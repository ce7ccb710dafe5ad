"""Linear time slab: coupled residual, Kronecker system, sequential stepping
and the splitting / defect-correction solve (oracle, test-only).

* Coupled residual, linear case (Sec. 2.2, residual R(Y) with f = K y - b,
  sign read as "+ F A2^T", consistent with Eq. matrix-fixed-point-equation):
      R(Y) = M Y A1^T + (K Y - B) A2^T - B0.
* Kronecker system, Eq. general-system-time-steps, with the column-stacking
  vec: [A1 (x) M + A2 (x) K] vec(Y) = [A2 (x) I] vec(B) + vec(B0), using
  (C (x) M) vec(Y) = vec(M Y C^T).
* Sequential stepping, Eq. stiffly-accurate-DIRK: one stage at a time,
  (M/tau + a_kk K) y_k = M y^n / tau - sum_{j<k} a_kj (K y_j - b_j) + a_kk b_k.
* Slab solve, Eq. matrix-fixed-point-equation written as defect correction:
      R = R(Y);  solve (alpha M + beta K) V = R;  Y <- Y - V,
  alpha = A1[0,0], beta = A2[0,0]; stop when every column k has
  ||R_k||_2 <= tol ||F_k||_2 with F = B A2^T + B0 (absolute if ||F_k|| = 0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from . import krylov


def coupled_residual(K, Mdiag, A1, A2, Y, B=None, B0=None):
    """R = M Y A1^T + (K Y - B) A2^T - B0 (B, B0 may be None = 0): the defect
    of Eq. general-system-time-steps in matrix form (column-stacking vec)."""
    KY = K @ Y
    if B is not None:
        KY = KY - B
    R = (Mdiag[:, None] * Y) @ A1.T + KY @ A2.T
    if B0 is not None:
        R = R - B0
    return R


def rhs_F(A2, B=None, B0=None, shape=None):
    """F = B A2^T + B0, the right-hand side of Eq. general-system-time-steps
    in matrix form."""
    F = np.zeros(shape) if B is None else B @ A2.T
    if B0 is not None:
        F = F + B0
    return F


def vec(X):
    """Column-stacking vec (Sec. 2.1, read as column stacking)."""
    return np.asarray(X).reshape(-1, order="F")


def unvec(x, n, s):
    """Inverse of the column-stacking vec of Eq. general-system-time-steps:
    x (N s) -> Y (N x s)."""
    return np.asarray(x).reshape(n, s, order="F")


def kron_operator(K, Mdiag, A1, A2):
    """Dense A1 (x) M + A2 (x) K (tiny grids only): the all-at-once operator
    of Eq. general-system-time-steps with column-stacking vec."""
    Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
    return np.kron(A1, np.diag(Mdiag)) + np.kron(A2, Kd)


def solve_all_at_once_dense(K, Mdiag, A1, A2, B=None, B0=None):
    """Dense LU solve of the Kronecker system (Eq. general-system-time-steps)."""
    n, s = K.shape[0], A1.shape[0]
    F = rhs_F(A2, B, B0, (n, s))
    y = np.linalg.solve(kron_operator(K, Mdiag, A1, A2), vec(F))
    return unvec(y, n, s)


def _gmres_solve(J, rhs, rtol):
    """x with ||J x - rhs|| <= rtol ||rhs|| by scipy's GMRES(200) with a
    Jacobi preconditioner; raises when it does not get there."""
    from scipy.sparse.linalg import LinearOperator, gmres
    d = J.diagonal()
    M = LinearOperator(J.shape, matvec=lambda x: x / d)
    x, info = gmres(J, rhs, rtol=rtol, atol=0.0, restart=200, maxiter=100, M=M)
    res = np.linalg.norm(J @ x - rhs)
    if info != 0 or res > 2.0 * rtol * np.linalg.norm(rhs):
        raise RuntimeError(f"stage solve did not reach rtol {rtol}: info {info}")
    return x


def sequential_dirk_linear(K, Mdiag, A, tau, y0, Bstages, rtol=None):
    """Step the stiffly accurate DIRK (Eq. stiffly-accurate-DIRK) one stage at
    a time. Bstages[:, g] is b(t) at global stage g (0-based, step-major).
    Returns the stage values (N x #stages); stages with a_kk = 0 are the
    explicit y^{(n,1)} = y^n.
    rtol None: each stage equation is solved by sparse LU (scipy splu). A
    float: by Jacobi-preconditioned GMRES (scipy) to that relative residual
    instead, for 3-D grids whose LU fill makes splu take minutes."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    N, G = Bstages.shape
    Y = np.zeros((N, G))
    yn = np.asarray(y0, dtype=np.float64).copy()
    Mdg = sp.diags(Mdiag)
    cache = {}
    for g in range(G):
        n, k = divmod(g, m)
        k += 1
        akk = A[k - 1, k - 1]
        rhs = Mdiag * yn / tau + akk * Bstages[:, g]
        for j in range(1, k):
            gj = n * m + j - 1
            rhs -= A[k - 1, j - 1] * (K @ Y[:, gj] - Bstages[:, gj])
        if akk == 0.0:
            Y[:, g] = yn
        elif rtol is None:
            if akk not in cache:
                cache[akk] = splu(sp.csc_matrix(Mdg / tau + akk * K))
            Y[:, g] = cache[akk].solve(rhs)
        else:
            Y[:, g] = _gmres_solve(sp.csr_matrix(Mdg / tau + akk * K), rhs, rtol)
        if k == m:
            yn = Y[:, g].copy()
    return Y


def slab_solve(K, Mdiag, A1, A2, B=None, B0=None, tol=1e-10, inner_tol=1e-2,
               precond="jacobi", restart=30, max_outer=200, inner_maxit=2000,
               exact_inner=False, Y0=None, narrow=False, solver="gmres"):
    """The method for a linear slab: defect correction around the splitting
    (Eq. matrix-splitting, Eq. matrix-fixed-point-equation) with a block GMRES
    inner solve on J = alpha M + beta K. Returns (Y, info).

    narrow: when A1 and A2 are lower triangular, the residual of column k
    depends on columns 0..k of Y only, so converged leading columns stay
    converged; the inner solve then takes only the trailing columns, the
    smallest power-of-two count that holds every unconverged one (the slab
    counterpart of dropping converged stages in Algorithm 1).

    solver: "gmres" (block GMRES(restart)), "cg" (block CG, symmetric
    positive definite J and preconditioner) or "bicgstab" (block BiCGStab,
    the paper's solver for the nonsymmetric linear problem)."""
    n, s = K.shape[0], A1.shape[0]
    alpha, beta, _, _ = _split(A1, A2)
    J = sp.csr_matrix(sp.diags(alpha * Mdiag) + beta * K)
    J.sort_indices()
    F = rhs_F(A2, B, B0, (n, s))
    Fn = np.linalg.norm(F, axis=0)
    thr = np.where(Fn > 0.0, tol * Fn, tol)
    Y = np.zeros((n, s)) if Y0 is None else np.array(Y0, dtype=np.float64)
    Pinv = krylov.make_preconditioner(J, precond)
    lu = splu(sp.csc_matrix(J)) if exact_inner else None
    hist, inner_its, col_steps = [], 0, 0
    for it in range(max_outer + 1):
        R = coupled_residual(K, Mdiag, A1, A2, Y, B, B0)
        rn = np.linalg.norm(R, axis=0)
        hist.append(rn / np.where(Fn > 0.0, Fn, 1.0))
        if np.all(rn <= thr) or it == max_outer:
            break
        c0 = 0
        if narrow and not np.any(np.triu(A1, 1)) and not np.any(np.triu(A2, 1)):
            lead = 0
            while lead < s and rn[lead] <= thr[lead]:
                lead += 1
            width = 1
            while width < s - lead:
                width *= 2
            c0 = s - width if width < s else 0
        if exact_inner:
            V = lu.solve(R[:, c0:])
        else:
            if solver == "cg":
                V, info = krylov.block_cg(lambda X: J @ X, Pinv, R[:, c0:], inner_tol,
                                          inner_maxit)
            elif solver == "bicgstab":
                V, info = krylov.block_bicgstab(lambda X: J @ X, Pinv, R[:, c0:], inner_tol,
                                                inner_maxit)
            else:
                V, info = krylov.block_gmres(lambda X: J @ X, Pinv, R[:, c0:], inner_tol,
                                             restart, inner_maxit)
            inner_its += info["iters"]
            col_steps += info["iters"] * (s - c0)
        Y[:, c0:] = Y[:, c0:] - V
    return Y, {"outer": len(hist) - 1, "inner": inner_its, "column_steps": col_steps,
               "relres": hist[-1],
               "history": hist, "converged": bool(np.all(rn <= thr))}


def slab_solve_global(K, Mdiag, A1, A2, B=None, B0=None, tol=1e-10, precond="jacobi",
                      restart=30, max_outer=200, maxit=100000, Y0=None, ortho="cgs2"):
    """The slab without the splitting (an extension beyond the paper): global
    GMRES(restart) (Jbilou, Messaoudi, Sadok 1999) on the coupled operator
    A(V) = M V A1^T + K V A2^T of Eq. general-system-time-steps, in the
    Frobenius inner product <X, Y> = trace(X^T Y), right-preconditioned column
    by column with the preconditioner of J = alpha M + beta K. Each cycle
    solves A(V) = R(Y) from V = 0 and sets Y <- Y - P(V); a cycle stops when
    its least-squares residual is below tol * min_k ||F_k|| (every column then
    meets its own tolerance) or after `restart` steps; the slab stops on the
    per-column test of slab_solve. Orthogonalisation in the Frobenius inner
    product: two classical Gram-Schmidt passes (ortho="cgs2") or modified
    Gram-Schmidt (ortho="mgs": one basis vector at a time, each product taken
    with the partly orthogonalised W). Returns (Y, info)."""
    n, s = K.shape[0], A1.shape[0]
    alpha, beta, _, _ = _split(A1, A2)
    J = sp.csr_matrix(sp.diags(alpha * Mdiag) + beta * K)
    J.sort_indices()
    Pinv = krylov.make_preconditioner(J, precond)
    F = rhs_F(A2, B, B0, (n, s))
    Fn = np.linalg.norm(F, axis=0)
    thr = np.where(Fn > 0.0, tol * Fn, tol)
    target = thr.min()
    Y = np.zeros((n, s)) if Y0 is None else np.array(Y0, dtype=np.float64)

    def A(V):
        return coupled_residual(K, Mdiag, A1, A2, V)

    def frob(X, Z):
        return float(np.sum(X * Z))

    hist, steps, cycles = [], 0, 0
    for it in range(max_outer + 1):
        R = coupled_residual(K, Mdiag, A1, A2, Y, B, B0)
        rn = np.linalg.norm(R, axis=0)
        hist.append(rn / np.where(Fn > 0.0, Fn, 1.0))
        if np.all(rn <= thr) or it == max_outer or steps >= maxit:
            break
        cycles += 1
        beta0 = np.sqrt(frob(R, R))
        V = [R / beta0]
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta0
        cs, sn = np.zeros(restart), np.zeros(restart)
        k = 0
        for j in range(restart):
            W = A(Pinv(V[j]))
            if ortho == "mgs":
                for i in range(j + 1):
                    H[i, j] = frob(V[i], W)
                    W = W - H[i, j] * V[i]
            else:
                for _ in range(2):                  # CGS2 in <., .>_F
                    h = np.array([frob(V[i], W) for i in range(j + 1)])
                    W = W - sum(h[i] * V[i] for i in range(j + 1))
                    H[:j + 1, j] += h
            H[j + 1, j] = np.sqrt(frob(W, W))
            V.append(W / H[j + 1, j] if H[j + 1, j] > 0.0 else np.zeros_like(W))
            for i in range(j):                      # earlier Givens rotations
                a, b = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
            r = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / r, H[j + 1, j] / r) if r > 0.0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = r, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            steps += 1
            k = j + 1
            if abs(g[j + 1]) <= target or steps >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        Z = sum(y[i] * V[i] for i in range(k))
        Y = Y - Pinv(Z)
    return Y, {"outer": len(hist) - 1, "inner": steps, "cycles": cycles, "relres": hist[-1],
               "history": hist, "converged": bool(np.all(rn <= thr))}


def _split(A1, A2):
    from .coupling import splitting
    return splitting(A1, A2)
