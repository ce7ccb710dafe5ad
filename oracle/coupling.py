"""Time-stepping matrices of the all-at-once DIRK system (oracle, test-only).

Sec. 2 ("Vectorized time integrators"):
  * stiffly accurate DIRK stage equations, Eq. stiffly-accurate-DIRK, read with
    the stage-k row index a_{k,j} (the printed a_{ij} is a typo);
  * single-step Kronecker form A1 = I/tau, A2 = A, B0 = (M y^n/tau, ...),
    Eq. general-system-time-steps;
  * elimination of an explicit first stage (a_11 = 0): the couplings
    a_{i1}(b^n - K y^n) move into B0 (Sec. 2.1, text after the Butcher tableau
    with A_impl);
  * s consecutive steps, Eq. time-stepping-matrices-multiple-parallel-time-steps:
    A1 = blockdiag(I_m)/tau with -1/tau in the last column of the previous
    block, A2 = blockdiag(A) (plus a_{i1} in the same places after an
    elimination), B0 non-zero only in the first m columns;
  * theta-method worked example, Example ex:time-stepping-matrices;
  * splitting A1 = alpha I + (A1 - alpha I), A2 = beta I + (A2 - beta I) with
    alpha = A1[0,0] (= 1/tau) and beta = A2[0,0] (top-left entry),
    Eq. matrix-splitting;
  * pipelined windows of Eq. matrix-equation-pipelining: the A1, A2 of a
    window that starts at an arbitrary stage, and which known quantities
    enter its B0.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------
# Butcher tableaux
# --------------------------------------------------------------------------
def implicit_euler():
    """Implicit Euler as a 1-stage stiffly accurate DIRK (Eq. stiffly-accurate-DIRK):
    A=[[1]], c=[1]."""
    return np.array([[1.0]]), np.array([1.0]), np.array([1.0])


def theta_method(theta: float):
    """Theta-method as a 2-stage DIRK with explicit first stage (Sec. 2.1,
    Example after the elimination): c=(0,1), A=[[0,0],[1-theta,theta]]."""
    A = np.array([[0.0, 0.0], [1.0 - theta, theta]])
    return A, A[-1].copy(), np.array([0.0, 1.0])


def sdirk2():
    """Two-stage L-stable SDIRK, gamma = 1 - 1/sqrt(2), stiffly accurate in the
    sense of Eq. stiffly-accurate-DIRK (the diffusion-reaction workload's
    integrator, standing in for Sec. 4.2's Crank-Nicolson)."""
    g = 1.0 - 1.0 / math.sqrt(2.0)
    A = np.array([[g, 0.0], [1.0 - g, g]])
    return A, A[-1].copy(), np.array([g, 1.0])


def is_stiffly_accurate(A, b) -> bool:
    """b_i = a_{m,i} for all i (Sec. 2)."""
    return bool(np.array_equal(np.asarray(b), np.asarray(A)[-1]))


# --------------------------------------------------------------------------
# One step, all stages (Eq. general-system-time-steps)
# --------------------------------------------------------------------------
def single_step_matrices(A, tau: float):
    """A1 = I_m / tau and A2 = A for the m stages of one step (Eq.
    general-system-time-steps with a single step)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    return np.eye(m) / tau, A.copy()


def eliminate_explicit_first_stage(A):
    """Split A with a_11 = 0 into (A_impl, e) with e_i = a_{i+1,1}, i=1..m-1
    (the elimination of the explicit first stage, Sec. 2.1).

    After the elimination the stage system has one stage less, operator
    (I/tau (x) M + A_impl (x) K), and B0 gains a_{i1}(b^n - K y^n) in row i.
    """
    A = np.asarray(A, dtype=np.float64)
    if A[0, 0] != 0.0 or np.any(A[0, 1:] != 0.0):
        raise ValueError("first stage is not explicit")
    return A[1:, 1:].copy(), A[1:, 0].copy()


# --------------------------------------------------------------------------
# s consecutive steps (Eq. time-stepping-matrices-multiple-parallel-time-steps)
# --------------------------------------------------------------------------
def multistep_matrices(A, s: int, tau: float, eliminate_first: bool = False):
    """Return (A1, A2, e) for s consecutive steps of the DIRK method A
    (Eq. time-stepping-matrices-multiple-parallel-time-steps).

    Block (n, n) of A1 is I_m'/tau, block (n, n-1) holds -1/tau in every row of
    its last column (y^{n} = y^{(n-1,m)} for stiffly accurate methods). A2 is
    blockdiag(A') with A' = A or A_impl; after an elimination the entries
    e_i = a_{i1} sit where A1 has its -1 entries. The same e gives the extra
    first-block B0 terms e_i (b^n - K y^n).
    """
    A = np.asarray(A, dtype=np.float64)
    if eliminate_first:
        Ap, e = eliminate_explicit_first_stage(A)
    else:
        Ap, e = A, np.zeros(A.shape[0])
    mp = Ap.shape[0]
    S = s * mp
    A1 = np.zeros((S, S))
    A2 = np.zeros((S, S))
    for n in range(s):
        blk = slice(n * mp, (n + 1) * mp)
        A1[blk, blk] = np.eye(mp) / tau
        A2[blk, blk] = Ap
        if n > 0:
            last_prev = n * mp - 1
            A1[blk, last_prev] = -1.0 / tau
            if eliminate_first:
                A2[blk, last_prev] = e
    return A1, A2, e


def theta_example_matrices(theta: float, s: int, tau: float):
    """Closed form of Example ex:time-stepping-matrices: A1 = (1/tau) lower
    bidiagonal (1, -1), A2 = lower bidiagonal (theta, 1-theta)."""
    A1 = (np.eye(s) - np.eye(s, k=-1)) / tau
    A2 = theta * np.eye(s) + (1.0 - theta) * np.eye(s, k=-1)
    return A1, A2


def theta_example_B0(theta, tau, Mdiag, K, yn, bn, s):
    """B0 = ((1/tau) M y^n - (1-theta)(K y^n - b^n), 0, ..., 0) of Example
    ex:time-stepping-matrices."""
    B0 = np.zeros((len(yn), s))
    B0[:, 0] = Mdiag * yn / tau - (1.0 - theta) * (K @ yn - bn)
    return B0


def splitting(A1, A2):
    """Eq. matrix-splitting: alpha = A1[0,0], beta = A2[0,0] and the parts
    A1 - alpha I, A2 - beta I moved to the right-hand side."""
    A1 = np.asarray(A1, dtype=np.float64)
    A2 = np.asarray(A2, dtype=np.float64)
    alpha = A1[0, 0]
    beta = A2[0, 0]
    s = A1.shape[0]
    return alpha, beta, A1 - alpha * np.eye(s), A2 - beta * np.eye(s)


# --------------------------------------------------------------------------
# Pipelined windows (Eq. matrix-equation-pipelining)
# --------------------------------------------------------------------------
def stage_of(g: int, m: int):
    """Global stage number g (0-based) -> (step n, stage k) with k in 1..m.

    This is the index map iota of Sec. 2.2 read as k = ((g) mod m) + 1 (the
    printed "k mod m" would give 0 at k = m)."""
    return g // m, g % m + 1


def window_matrices(A, c, tau: float, g0: int, s: int):
    """A1, A2 (s x s) and the B0 recipe (Eq. matrix-equation-pipelining,
    Algorithm 1) of the window of s consecutive stages
    starting at global stage g0 (0-based) of the stiffly accurate DIRK (A, c).

    Stage (n, k) reads (1/tau)(M(y^{(n,k)}) - M(y^n)) + sum_{j<=k} a_kj
    f(t^{(n,j)}, y^{(n,j)}) = 0, with y^n = y^{(n-1,m)} (or y_0 for n = 0).
    A coupling to a stage inside the window becomes an entry of A1 (the mass
    term) or A2 (the f terms). A coupling to an earlier, already converged
    stage is moved to B0, which is returned as a list of terms
        (column i, "mass", global stage of y^n, coefficient 1/tau)
        (column i, "f", global stage (n, j), coefficient -a_kj)
    where global stage -1 stands for the initial value y_0.
    Returns (A1, A2, terms, times) with times[i] = t^n + c_k tau relative to
    t = 0 at step 0.
    """
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    A1 = np.zeros((s, s))
    A2 = np.zeros((s, s))
    terms = []
    times = np.zeros(s)
    for i in range(s):
        g = g0 + i
        n, k = stage_of(g, m)
        times[i] = (n + c[k - 1]) * tau
        A1[i, i] += 1.0 / tau
        gprev = n * m - 1            # y^n = last stage of step n-1
        if gprev >= g0:
            A1[i, gprev - g0] += -1.0 / tau
        else:
            terms.append((i, "mass", gprev, 1.0 / tau))
        for j in range(1, k + 1):
            gj = n * m + j - 1
            if gj >= g0:
                A2[i, gj - g0] += A[k - 1, j - 1]
            elif A[k - 1, j - 1] != 0.0:
                terms.append((i, "f", gj, -A[k - 1, j - 1]))
    return A1, A2, terms, times


def shift(Y):
    """shift((Y_1,...,Y_s)) = (Y_2,...,Y_s,Y_s), Sec. 2.2 (Eq. shift)."""
    Y = np.asarray(Y)
    return np.concatenate([Y[:, 1:], Y[:, -1:]], axis=1)
