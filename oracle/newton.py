"""Nonlinear time stepping (oracle, test-only).

Semi-discrete form M(y)' + f(t, y) = 0 with f(t,y) = K[y] y - b(t)
(Sec. 2.2; a state-dependent mass M(y) = theta(psi) for Richards, Remark
"Additional Nonlinearity").

* `sequential_dirk_newton`: the plain definition. The stiffly accurate DIRK
  stage equations of Eq. stiffly-accurate-DIRK (K -> K[y]) are solved one
  stage after the other with full Newton,
      G(y) = (1/tau)(M(y) - M(y^n)) + sum_{j<k} a_kj f_j + a_kk f(t_k, y) = 0,
  to a relative residual of `tol`.
* `pipelined_block_newton`: Algorithm 1 ("Block Krylov Time Stepping with
  Pipelining"). A window of s consecutive stages starts at (y_0,...,y_0);
  for each window the residual
      R(Y) = M(Y) A1^T + F(T, Y) A2^T - B0        (sign read as "+ F A2^T")
  of Eq. matrix-equation-pipelining is driven to ||R_0|| <= eps ||F_0|| in
  column 0 (F_0 = B0_0) by simplified Newton steps with the first column's
  Jacobian
      J = (1/tau) M'(Y_0) + a_kk Df(t_0, Y_0),
  each solving J V = R for all s columns with block GMRES; then the window is
  shifted (Eq. shift) by one stage.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from . import coupling, fv, krylov


class LinearProblem:
    """M y' + K y - b(t) = 0 with diagonal M: Eq. problem with f linear."""

    def __init__(self, K, Mdiag, b):
        self.K, self.Mdiag, self.b = K, np.asarray(Mdiag, dtype=np.float64), b

    def mass(self, y):
        return self.Mdiag * y

    def dmass(self, y):
        return self.Mdiag.copy()

    def f(self, t, y):
        return self.K @ y - self.b(t)

    def jac(self, t, y):
        return sp.csr_matrix(self.K)


class DiffReactProblem:
    """u_t = div((1+u^2) grad u) + u(1-u) + src(t), M = I (oracle.fv): the
    diffusion-reaction problem of Sec. 4.2."""

    def __init__(self, dims):
        self.dims = dims

    def mass(self, y):
        return y.copy()

    def dmass(self, y):
        return np.ones_like(y)

    def f(self, t, y):
        return fv.diffreact_f(self.dims, t, y)

    def jac(self, t, y):
        return fv.diffreact_jacobian(self.dims, t, y)


class RichardsProblem:
    """d/dt theta(psi) - div(K(psi) grad(psi + z)) = 0 (oracle.fv): Richards'
    equation of Sec. 4.3 (mass term M(y) of Sec. 2.2)."""

    def __init__(self, dims, Ks, vg, dt_D):
        self.dims, self.Ks, self.vg, self.dt_D = dims, Ks, vg, dt_D

    def mass(self, y):
        return self.vg.theta(y)

    def dmass(self, y):
        return self.vg.dtheta(y)

    def f(self, t, y):
        return fv.richards_f(self.dims, t, y, self.Ks, self.vg, self.dt_D)

    def jac(self, t, y):
        return fv.richards_jacobian(self.dims, t, y, self.Ks, self.vg, self.dt_D)

    def jac_frozen(self, t, y):
        """Flux operator with the conductivities frozen at y (L-scheme)."""
        return fv.richards_jacobian(self.dims, t, y, self.Ks, self.vg, self.dt_D, frozen=True)


def sequential_dirk_newton(prob, A, c, tau, y0, nstages, tol=1e-13, maxit=50):
    """Plain definition: one stage at a time, full Newton, sparse direct solves.
    Returns (stages N x nstages, newton iterations per stage)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    y0 = np.asarray(y0, dtype=np.float64)
    Y = np.zeros((len(y0), nstages))
    fs = np.zeros_like(Y)
    its = []
    yn = y0.copy()
    for g in range(nstages):
        n, k = coupling.stage_of(g, m)
        t = (n + c[k - 1]) * tau
        known = prob.mass(yn) / tau
        for j in range(1, k):
            known = known - A[k - 1, j - 1] * fs[:, n * m + j - 1]
        akk = A[k - 1, k - 1]
        y = (Y[:, g - 1] if g > 0 else yn).copy()
        scale = max(np.linalg.norm(known), 1e-300)
        for it in range(maxit + 1):
            Gv = prob.mass(y) / tau + akk * prob.f(t, y) - known
            if np.linalg.norm(Gv) <= tol * scale:
                break
            Jm = sp.diags(prob.dmass(y) / tau) + akk * prob.jac(t, y)
            y = y - splu(sp.csc_matrix(Jm)).solve(Gv)
        its.append(it)
        Y[:, g] = y
        fs[:, g] = prob.f(t, y)
        if k == m:
            yn = y.copy()
    return Y, its


def window_B0(prob, terms, stages, fvals, y0, s):
    """B0 of a window (Eq. matrix-equation-pipelining) from the recipe of
    coupling.window_matrices."""
    n = len(y0)
    B0 = np.zeros((n, s))
    for i, kind, g, coef in terms:
        if kind == "mass":
            y = y0 if g < 0 else stages[g]
            B0[:, i] += coef * prob.mass(y)
        else:
            B0[:, i] += coef * fvals[g]
    return B0


def window_residual(prob, A1, A2, times, Y, B0):
    """R(Y) = M(Y) A1^T + F(T, Y) A2^T - B0 (Eq. matrix-equation-pipelining)."""
    s = Y.shape[1]
    MY = np.column_stack([prob.mass(Y[:, i]) for i in range(s)])
    FY = np.column_stack([prob.f(times[i], Y[:, i]) for i in range(s)])
    return MY @ A1.T + FY @ A2.T - B0


def linearisation(prob, alpha, beta, t, y, lscheme_L=None):
    """Matrix of one outer iteration: the simplified-Newton Jacobian
    alpha M'(y) + beta Df(t, y) (Algorithm 1), or with lscheme_L the L-scheme
    of Sec. 4.3 (Richards): M' replaced by the constant L, the conductivities
    frozen at y: alpha L I + beta A(y)."""
    if lscheme_L:
        J = sp.identity(len(y)) * (alpha * lscheme_L) + beta * prob.jac_frozen(t, y)
    else:
        J = sp.diags(alpha * prob.dmass(y)) + beta * prob.jac(t, y)
    J = sp.csr_matrix(J)
    J.sort_indices()
    return J


def pipelined_block_newton(prob, A, c, tau, y0, nstages, s, tol=1e-8, inner_tol=1e-5,
                           precond="ilu0", restart=30, max_newton=50, inner_maxit=1000,
                           max_step=None, lscheme_L=None, solver="gmres"):
    """Algorithm 1 over `nstages` global stages with a window of s stages.
    Returns (stages N x nstages, stats dict).

    solver: the inner block solver, "gmres" (block GMRES(restart)), "cg"
    (block CG: the L-scheme matrix of Richards' equation and its ILU(0) are
    symmetric positive definite) or "bicgstab" (block BiCGStab).

    max_step (reading, the paper gives no globalisation): when set, column k
    of each Newton update V is scaled by min(1, max_step / max_r |V_rk|). The
    trailing columns of a window take chord steps with the first column's
    Jacobian; for Richards' equation they can otherwise leave the physical
    range of heads and poison later windows."""
    y0 = np.asarray(y0, dtype=np.float64)
    N = len(y0)
    Y = np.repeat(y0[:, None], s, axis=1)
    stages, fvals = {}, {}
    newton_its, inner_its = [], 0
    for g0 in range(nstages):
        A1, A2, terms, times = coupling.window_matrices(A, c, tau, g0, s)
        B0 = window_B0(prob, terms, stages, fvals, y0, s)
        F0 = np.linalg.norm(B0[:, 0])
        thr = tol * (F0 if F0 > 0.0 else 1.0)
        alpha, beta = A1[0, 0], A2[0, 0]
        for it in range(max_newton + 1):
            R = window_residual(prob, A1, A2, times, Y, B0)
            if np.linalg.norm(R[:, 0]) <= thr or it == max_newton:
                break
            J = linearisation(prob, alpha, beta, times[0], Y[:, 0], lscheme_L)
            Pinv = krylov.make_preconditioner(J, precond)
            if solver == "cg":
                V, info = krylov.block_cg(lambda X: J @ X, Pinv, R, inner_tol, inner_maxit)
            elif solver == "bicgstab":
                V, info = krylov.block_bicgstab(lambda X: J @ X, Pinv, R, inner_tol,
                                                inner_maxit)
            else:
                V, info = krylov.block_gmres(lambda X: J @ X, Pinv, R, inner_tol, restart,
                                             inner_maxit)
            inner_its += info["iters"]
            if max_step:
                vmax = np.max(np.abs(V), axis=0)
                V = V * np.minimum(1.0, max_step / np.maximum(vmax, 1e-300))
            Y = Y - V
        newton_its.append(it)
        stages[g0] = Y[:, 0].copy()
        fvals[g0] = prob.f(times[0], Y[:, 0])
        Y = coupling.shift(Y)
    out = np.column_stack([stages[g] for g in range(nstages)])
    return out, {"newton": newton_its, "inner": inner_its}
