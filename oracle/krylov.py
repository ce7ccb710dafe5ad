"""Block Krylov pieces of the vectorised solve (oracle, test-only).

The paper solves the matrix equation (1/tau M + beta K) Y = RHS of
Eq. matrix-fixed-point-equation with a block Krylov method (Sec. 2.1, and
Sec. 1 "AX = B ... Block Krylov methods"); it is silent on
orthogonalisation and preconditioning side. The readings used here and on
the device are:
  * block GMRES with restart m (default 30), right preconditioning, X0 = 0;
  * block classical Gram-Schmidt applied twice (BCGS2) against the basis;
  * CholQR2 for the new basis block: G = W^T W, upper Cholesky G = R^T R in
    natural column order, W <- W R^{-1}, done twice; a column whose Cholesky
    pivot falls to <= defl * G_kk (or G_kk == 0) is deflated: its row of R is
    zero and its basis column is zero;
  * the block Hessenberg least-squares problem is reduced by Householder
    reflectors of length s+1, one per column; the per-column residual
    estimates are the norms of the last s rows of the rotated right-hand side;
  * Jacobi: P^{-1} = diag(J)^{-1}; ILU(0): incomplete LU in natural order on
    the pattern of J (IKJ variant), applied by forward / backward substitution;
  * block CG (symmetric systems) re-orthonormalises its search block every
    iteration; block BiCGStab (nonsymmetric systems) deflates the right-hand
    side block once, by CholQR2, before it starts.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


# --------------------------------------------------------------------------
# CholQR with deflation
# --------------------------------------------------------------------------
def cholesky_deflating(G, defl):
    """Upper R with G = R^T R (natural order; the paper is silent on
    orthogonalisation, this is the module's CholQR reading). Deflated rows
    are zero.
    Returns (R, deflated mask)."""
    s = G.shape[0]
    R = np.zeros_like(G)
    dead = np.zeros(s, dtype=bool)
    for k in range(s):
        d = G[k, k] - np.dot(R[:k, k], R[:k, k])
        if G[k, k] <= 0.0 or d <= defl * G[k, k]:
            dead[k] = True
            continue
        R[k, k] = np.sqrt(d)
        for j in range(k + 1, s):
            R[k, j] = (G[k, j] - np.dot(R[:k, k], R[:k, j])) / R[k, k]
    return R, dead


def cholqr(W, defl=1e-14):
    """One CholQR pass (module reading): W = Q R, Q = W R^{-1} column by column."""
    G = W.T @ W
    R, dead = cholesky_deflating(G, defl)
    s = W.shape[1]
    Q = np.zeros_like(W)
    for k in range(s):
        if dead[k]:
            continue
        Q[:, k] = (W[:, k] - Q[:, :k] @ R[:k, k]) / R[k, k]
    return Q, R


def cholqr2(W, defl=1e-14):
    """CholQR applied twice (module reading); R = R2 R1."""
    Q1, R1 = cholqr(W, defl)
    Q, R2 = cholqr(Q1, defl)
    return Q, R2 @ R1


def bcgs2(Vs, W):
    """Two passes of block classical Gram-Schmidt (module reading) of W against
    the blocks Vs.
    Returns (W_orth, H) with W = W_orth + [V] H."""
    Vm = np.hstack(Vs)
    H = np.zeros((Vm.shape[1], W.shape[1]))
    for _ in range(2):
        Hp = Vm.T @ W
        W = W - Vm @ Hp
        H = H + Hp
    return W, H


# --------------------------------------------------------------------------
# Householder reduction of the block Hessenberg matrix
# --------------------------------------------------------------------------
def householder(x):
    """Householder reflector (textbook; module reading for the block
    Hessenberg least squares): unit v and beta with (I - 2 v v^T) x =
    beta e_1; v = 0 if x = 0."""
    nx = np.linalg.norm(x)
    if nx == 0.0:
        return np.zeros_like(x), 0.0
    beta = -nx if x[0] >= 0.0 else nx
    v = x.copy()
    v[0] -= beta
    v /= np.linalg.norm(v)
    return v, beta


def apply_reflector(v, Yblk):
    """Yblk <- (I - 2 v v^T) Yblk (rows of Yblk match v); textbook."""
    Yblk -= 2.0 * np.outer(v, v @ Yblk)


# --------------------------------------------------------------------------
# Block GMRES(m), right preconditioned
# --------------------------------------------------------------------------
def block_gmres(apply_J, apply_Pinv, R, tol, restart=30, maxit=1000, defl=1e-14):
    """Block GMRES(restart) (the block Krylov solve of Eq.
    matrix-fixed-point-equation, Sec. 2.1, with the module's readings):
    solve J X = R for X (N x s) to per-column relative residual `tol`.

    apply_J(X) and apply_Pinv(X) act on N x s blocks. Returns (X, info) with
    info = {iters, restarts, est (final per-column estimates), converged}.
    """
    N, s = R.shape
    X = np.zeros_like(R)
    r0 = np.linalg.norm(R, axis=0)
    target = tol * r0
    its = 0
    cycles = 0
    Rc = R.copy()
    est = r0.copy()
    converged = bool(np.all(r0 == 0.0))
    while not converged and its < maxit:
        cycles += 1
        V0, S = cholqr2(Rc, defl)
        V = [V0]
        m = restart
        Hb = np.zeros(((m + 1) * s, m * s))
        G = np.zeros(((m + 1) * s, s))
        G[:s] = S
        refl = []
        j_done = 0
        for j in range(m):
            W = apply_J(apply_Pinv(V[j]))
            W, H = bcgs2(V, W)
            Vn, Rn = cholqr2(W, defl)
            col = np.zeros(((m + 1) * s, s))
            col[:(j + 1) * s] = H
            col[(j + 1) * s:(j + 2) * s] = Rn
            for c, v in enumerate(refl):                 # earlier reflectors
                apply_reflector(v, col[c:c + s + 1])
            for l in range(s):                           # this block's columns
                c = j * s + l
                v, beta = householder(col[c:c + s + 1, l].copy())
                if l + 1 < s:
                    apply_reflector(v, col[c:c + s + 1, l + 1:])
                col[c, l] = beta
                col[c + 1:c + s + 1, l] = 0.0
                apply_reflector(v, G[c:c + s + 1])
                refl.append(v)
            Hb[:, j * s:(j + 1) * s] = col
            V.append(Vn)
            its += 1
            j_done = j + 1
            est = np.linalg.norm(G[(j + 1) * s:(j + 2) * s], axis=0)
            if np.all(est <= target) or its >= maxit:
                break
        k = j_done * s
        Rt = Hb[:k, :k]
        Y = np.zeros((k, s))
        scale = np.max(np.abs(np.diag(Rt))) if k else 0.0
        for i in range(k - 1, -1, -1):                  # back substitution
            if abs(Rt[i, i]) <= 1e-300 + 1e-14 * scale:
                continue
            Y[i] = (G[i] - Rt[i, i + 1:] @ Y[i + 1:]) / Rt[i, i]
        X = X + apply_Pinv(np.hstack(V[:j_done]) @ Y)
        converged = bool(np.all(est <= target))
        if not converged:
            Rc = R - apply_J(X)
    return X, {"iters": its, "restarts": cycles, "est": est, "converged": converged}


# --------------------------------------------------------------------------
# Preconditioners
# --------------------------------------------------------------------------
def jacobi(J):
    """Jacobi preconditioner (the workloads' choice for the 2-D linear slab):
    P^{-1} X = diag(J)^{-1} X."""
    d = J.diagonal().copy()
    return lambda X: X / d[:, None]


def ilu0(J):
    """ILU(0) (the workloads' preconditioner; the paper uses AMG, out of
    scope) of CSR J in natural order (IKJ): for each row i and each k < i in
    its pattern, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for j > k in both
    rows' patterns. Returns (L unit lower, U upper) as CSR."""
    J = sp.csr_matrix(J, dtype=np.float64, copy=True)
    J.sort_indices()
    ptr, col, val = J.indptr, J.indices, J.data.copy()
    n = J.shape[0]
    diag = np.empty(n, dtype=np.int64)
    for i in range(n):
        pos = np.searchsorted(col[ptr[i]:ptr[i + 1]], i)
        diag[i] = ptr[i] + pos
    for i in range(n):
        a, b = ptr[i], ptr[i + 1]
        where = {int(col[p]): p for p in range(a, b)}
        for p in range(a, b):
            k = int(col[p])
            if k >= i:
                break
            val[p] /= val[diag[k]]
            for q in range(diag[k] + 1, ptr[k + 1]):
                j = int(col[q])
                t = where.get(j)
                if t is not None:
                    val[t] -= val[p] * val[q]
    F = sp.csr_matrix((val, col.copy(), ptr.copy()), shape=J.shape)
    L = sp.tril(F, k=-1, format="csr") + sp.identity(n, format="csr")
    U = sp.triu(F, k=0, format="csr")
    L.sort_indices()
    U.sort_indices()
    return L, U


def ilu0_apply(L, U):
    """P^{-1} X = U^{-1} L^{-1} X for the ILU(0) factors (forward, then
    backward substitution; textbook)."""
    def f(X):
        Y = spsolve_triangular(L, X, lower=True, unit_diagonal=True)
        return spsolve_triangular(U, Y, lower=False)
    return f


def make_preconditioner(J, kind):
    """P^{-1} as a function of a block X: "none", "jacobi" or "ilu0" (the
    module's preconditioner readings)."""
    if kind == "none":
        return lambda X: X.copy()
    if kind == "jacobi":
        return jacobi(J)
    if kind == "ilu0":
        return ilu0_apply(*ilu0(J))
    raise ValueError(kind)


# --------------------------------------------------------------------------
# ILU(0) of a grid-stencil matrix, by hyperplanes (for large grids)
# --------------------------------------------------------------------------
def _stencil_offsets(dims):
    """Index offsets of the x, y, z neighbours, for the axes of extent > 1."""
    nx, ny, nz = dims
    return tuple(o for o, m in ((1, nx), (nx, ny), (nx * ny, nz)) if m > 1)


def ilu0_stencil(dims, J):
    """ILU(0) in natural order of a matrix whose pattern is (a subset of) the
    3/5/7-point stencil of the grid dims = (nx, ny, nz), cell x + nx (y + ny z).

    For such a pattern the IKJ elimination of `ilu0` changes only the
    diagonal: the product l_ik u_kj of a lower neighbour k of i and an upper
    neighbour j of k lies in row i's pattern only for j = i (two distinct
    stencil offsets never differ by a third between true grid neighbours).
    Hence U keeps J's upper entries, l_ik = a_ik / d_k and
        d_i = a_ii - sum_{k lower neighbour of i} a_ik a_ki / d_k.
    Cells on one hyperplane x + y + z = const depend only on the previous
    hyperplane, so each plane is one vectorised step. Pinned against `ilu0`
    on small grids. Returns (d, lower, upper): lower[o][i] = a_{i,i-o},
    upper[o][i] = a_{i,i+o} for the offsets o of the grid (0 where absent)."""
    J = sp.coo_matrix(J)
    n = int(np.prod(dims))
    offs = _stencil_offsets(dims)
    lower = {o: np.zeros(n) for o in offs}
    upper = {o: np.zeros(n) for o in offs}
    diag = np.zeros(n)
    delta = J.col.astype(np.int64) - J.row.astype(np.int64)
    np.add.at(diag, J.row[delta == 0], J.data[delta == 0])
    for o in offs:
        m = delta == -o
        np.add.at(lower[o], J.row[m], J.data[m])
        m = delta == o
        np.add.at(upper[o], J.row[m], J.data[m])
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    level = (x + y + z).ravel()
    d = diag.copy()
    for L in range(1, int(level.max()) + 1 if n else 0):
        rows = np.nonzero(level == L)[0]
        acc = np.zeros(len(rows))
        for o in offs:
            a_ik = lower[o][rows]
            has = a_ik != 0.0
            k = rows[has] - o
            acc[has] += a_ik[has] * upper[o][k] / d[k]
        d[rows] = diag[rows] - acc
    return d, lower, upper


def ilu0_stencil_apply(dims, fac, X):
    """P^{-1} X = U^{-1} L^{-1} X for the factors of `ilu0_stencil`, plane by
    plane (forward over increasing x + y + z, backward over decreasing)."""
    d, lower, upper = fac
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    level = (x + y + z).ravel()
    nlev = int(level.max()) + 1 if n else 0
    planes = [np.nonzero(level == L)[0] for L in range(nlev)]
    offs = _stencil_offsets(dims)
    Y = X.copy()
    for rows in planes:                          # L y = x, unit lower
        for o in offs:
            l = lower[o][rows]
            has = l != 0.0
            k = rows[has] - o
            Y[rows[has]] -= (l[has] / d[k])[:, None] * Y[k]
    Z = Y.copy()
    for rows in reversed(planes):                # U z = y
        for o in offs:
            u = upper[o][rows]
            has = u != 0.0
            j = rows[has] + o
            Z[rows[has]] -= u[has][:, None] * Z[j]
        Z[rows] /= d[rows][:, None]
    return Z


# --------------------------------------------------------------------------
# Block conjugate gradients (the paper's solver for symmetric systems)
# --------------------------------------------------------------------------
def _spd_pinv_apply(G, rhs, defl):
    """(G)^+ rhs for a symmetric positive semi-definite s x s G, read as the
    inverse of G on its active columns (reading of the breakdown-free block
    CG): the deflating Cholesky test decides which columns are dependent; the
    result solves G[a, a] x_a = rhs[a] on the active set a and is zero on the
    deflated rows."""
    _, dead = cholesky_deflating(G, defl)
    act = np.flatnonzero(~np.asarray(dead, dtype=bool))
    out = np.zeros((G.shape[0],) + rhs.shape[1:])
    if act.size:
        out[act] = np.linalg.solve(G[np.ix_(act, act)], rhs[act])
    return out


def block_cg(apply_J, apply_Minv, R, tol, maxit=1000, defl=1e-14):
    """Preconditioned block CG (Sec. 4.2 and 4.3 solve with a block CG) for
    symmetric positive definite J and M,
    breakdown-free form: the search block is orthonormalised (CholQR2 with
    deflation) every iteration, so dependent or converged columns drop out
    instead of making P^T J P singular:
        Z = M^-1 R;  P = orth(Z)
        repeat: Q = J P;  a = (P^T Q)^+ P^T R;  X += P a;  R -= Q a
                Z = M^-1 R;  b = -(P^T Q)^+ Q^T Z;  P = orth(Z + P b)
    until every column satisfies ||R_k|| <= tol ||R0_k||. X0 = 0.
    Returns (X, info) with info = {iters, est, converged}."""
    N, s = R.shape
    X = np.zeros_like(R)
    r0 = np.linalg.norm(R, axis=0)
    target = tol * r0
    Rc = R.copy()
    est = r0.copy()
    if np.all(r0 == 0.0):
        return X, {"iters": 0, "est": est, "converged": True}
    P, _ = cholqr2(apply_Minv(Rc), defl)
    its = 0
    while its < maxit:
        Q = apply_J(P)
        G = P.T @ Q
        a = _spd_pinv_apply(G, P.T @ Rc, defl)
        X = X + P @ a
        Rc = Rc - Q @ a
        its += 1
        est = np.linalg.norm(Rc, axis=0)
        if np.all(est <= target):
            break
        Z = apply_Minv(Rc)
        b = -_spd_pinv_apply(G, Q.T @ Z, defl)
        P, _ = cholqr2(Z + P @ b, defl)
    return X, {"iters": its, "est": est, "converged": bool(np.all(est <= target))}


# --------------------------------------------------------------------------
# Block BiCGStab (the paper's solver for the linear convection-diffusion
# problem, Sec. 4.1)
# --------------------------------------------------------------------------
def _solve_active(G, rhs, active):
    """G^{-1} rhs on the active rows and columns of the s x s G; the rows of
    inactive (deflated) columns are zero."""
    out = np.zeros((G.shape[0], rhs.shape[1]))
    a = np.flatnonzero(active)
    if a.size:
        out[a] = np.linalg.solve(G[np.ix_(a, a)], rhs[a])
    return out


def block_bicgstab(apply_J, apply_Minv, R, tol, maxit=1000, defl=1e-14, record=None):
    """Right-preconditioned block BiCGStab (Guennouni, Jbilou and Sadok, "A
    block version of BiCGSTAB for linear systems with multiple right-hand
    sides", ETNA 16, 2003) for a nonsymmetric J, X0 = 0.

    The published method has no treatment of dependent right-hand sides, for
    which the s x s matrices Rt^T V are singular from the start. The reading
    here deflates once, up front: R = Q0 C by CholQR2 with deflation, the
    iteration solves J Xh = Q0 with the shadow block Rt = Q0 (deflated
    columns of Q0 are zero and stay zero; the s x s solves act on the active
    columns only), and X = Xh C:
        Rh = P = Q0
        repeat: Ph = M^-1 P;  V = J Ph;  alpha = (Rt^T V)^-1 Rt^T Rh
                S = Rh - V alpha;  Sh = M^-1 S;  T = J Sh
                omega = <T, S>_F / <T, T>_F
                Xh += Ph alpha + omega Sh;  Rh = S - omega T
                stop when every column of Rh C is <= tol ||R_k||
                beta = -(Rt^T V)^-1 Rt^T T;  P = Rh + (P - omega V) beta
    `record`, a list, receives per iteration the quantities that define
    alpha, omega and beta (Rt^T S, <T, S - omega T>_F, Rt^T (T + V beta)),
    all zero in exact arithmetic. Returns (X, info) with info = {iters, est,
    converged}."""
    N, s = R.shape
    r0 = np.linalg.norm(R, axis=0)
    target = tol * r0
    if np.all(r0 == 0.0):
        return np.zeros_like(R), {"iters": 0, "est": r0, "converged": True}
    Q0, C = cholqr2(R, defl)
    active = np.diag(C) != 0.0
    Rt = Q0
    Rh = Q0.copy()
    P = Q0.copy()
    Xh = np.zeros_like(R)
    est = r0.copy()
    its = 0
    while its < maxit:
        Ph = apply_Minv(P)
        V = apply_J(Ph)
        G = Rt.T @ V
        alpha = _solve_active(G, Rt.T @ Rh, active)
        S = Rh - V @ alpha
        Sh = apply_Minv(S)
        T = apply_J(Sh)
        tt = float(np.sum(T * T))
        omega = float(np.sum(T * S)) / tt if tt > 0.0 else 0.0
        Xh = Xh + Ph @ alpha + omega * Sh
        Rh = S - omega * T
        its += 1
        est = np.linalg.norm(Rh @ C, axis=0)
        if not np.all(np.isfinite(est)) or np.all(est <= target):
            if record is not None:
                record.append({"RtS": Rt.T @ S, "omega_orth": float(np.sum(T * Rh))})
            break
        beta = -_solve_active(G, Rt.T @ T, active)
        if record is not None:
            record.append({"RtS": Rt.T @ S, "omega_orth": float(np.sum(T * Rh)),
                           "RtTVb": Rt.T @ (T + V @ beta)})
        P = Rh + (P - omega * V) @ beta
    return Xh @ C, {"iters": its, "est": est,
                    "converged": bool(np.all(est <= target))}
