"""Cell-centred finite-volume operators on the unit square / cube (oracle).

The paper discretises with CCFV and Q1 FE (Sec. 4); the synthetic workloads
here use CCFV on [0,1]^d with h = 1/nx for every direction, natural (x-fastest)
cell numbering r = i + nx*(j + ny*k), and equations per unit volume (M = I for
the linear and diffusion-reaction problems). The discretisation choices the
paper does not fix are:
  * diffusion faces use the harmonic mean of the two cell coefficients;
  * a homogeneous Dirichlet boundary face is a ghost at distance h/2
    (coefficient 2 D / h^2);
  * convection is first-order upwind on the face-normal velocity, with zero
    inflow value and free outflow on the boundary;
  * diffusion-reaction: arithmetic face mean of (1 + u^2), zero-flux Neumann;
  * Richards: face conductivity = harmonic mean of K_S times the relative
    permeability of the upwind cell by total head psi + z (tie: the cell with
    the lower index), van Genuchten-Mualem relations of Eq. RelationshipsThetaK
    read literally with theta/theta_S.
Everything returns scipy CSR matrices with sorted column indices, no explicit
zeros for absent neighbours.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def grid_index(dims):
    """Natural x-fastest cell numbering of an nx x ny x nz grid, as an array
    of shape (nz, ny, nx) (the matrix-based FV setting of Sec. 1)."""
    nx, ny, nz = dims
    return np.arange(nx * ny * nz).reshape(nz, ny, nx)


def _faces(dims):
    """Yield (d, P, Q) arrays of interior faces with Q = P + e_d."""
    idx = grid_index(dims)
    nx, ny, nz = dims
    if nx > 1:
        yield 0, idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()
    if ny > 1:
        yield 1, idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()
    if nz > 1:
        yield 2, idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()


def _boundary(dims):
    """Yield (d, sign, P) for boundary faces with outward normal sign * e_d."""
    idx = grid_index(dims)
    nx, ny, nz = dims
    if nx > 1:
        yield 0, -1, idx[:, :, 0].ravel()
        yield 0, +1, idx[:, :, -1].ravel()
    if ny > 1:
        yield 1, -1, idx[:, 0, :].ravel()
        yield 1, +1, idx[:, -1, :].ravel()
    if nz > 1:
        yield 2, -1, idx[0, :, :].ravel()
        yield 2, +1, idx[-1, :, :].ravel()


def _csr(rows, cols, vals, n):
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def pattern(dims):
    """Sparsity pattern of the 5- / 7-point stencil (all ones): the pattern K
    shares with every Jacobian of Sec. 2.2."""
    n = int(np.prod(dims))
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.ones(n)]
    for _, P, Q in _faces(dims):
        rows += [P, Q]
        cols += [Q, P]
        vals += [np.ones(len(P)), np.ones(len(P))]
    return _csr(rows, cols, vals, n)


# --------------------------------------------------------------------------
# Linear convection-diffusion: K u = -div(D grad u) + div(v u)
# --------------------------------------------------------------------------
def convdiff_matrix(dims, D, velocity):
    """Stiffness matrix K of -div(D grad u) + div(v u) on [0,1]^d (the linear
    problem of Sec. 4.1; the paper gives no FV details, so the cell-centred
    scheme below is this module's reading).

    D has shape (nz, ny, nx); velocity is (vx, vy, vz), constant. Homogeneous
    Dirichlet on every boundary face for diffusion, upwind convection with zero
    inflow value.
    """
    nx = dims[0]
    h = 1.0 / nx
    n = int(np.prod(dims))
    Dr = np.asarray(D, dtype=np.float64).ravel()
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r)
        cols.append(c)
        vals.append(v)

    for d, P, Q in _faces(dims):
        Df = 2.0 * Dr[P] * Dr[Q] / (Dr[P] + Dr[Q])
        g = Df / h**2
        add(P, P, g); add(P, Q, -g); add(Q, Q, g); add(Q, P, -g)
        vn = velocity[d]
        if vn > 0.0:          # flux P -> Q equals vn * u_P
            w = np.full(len(P), vn / h)
            add(P, P, w); add(Q, P, -w)
        elif vn < 0.0:        # flux P -> Q equals vn * u_Q
            w = np.full(len(P), vn / h)
            add(P, Q, w); add(Q, Q, -w)
    for d, sgn, P in _boundary(dims):
        add(P, P, 2.0 * Dr[P] / h**2)
        vn = sgn * velocity[d]
        if vn > 0.0:          # outflow through the boundary
            add(P, P, np.full(len(P), vn / h))
    return _csr(rows, cols, vals, n)


# --------------------------------------------------------------------------
# Nonlinear diffusion-reaction: u_t = div((1+u^2) grad u) + u(1-u) + src
# --------------------------------------------------------------------------
def circle_source(dims, t):
    """Moving-circle source of Sec. 4.2: -0.1 inside the disc of radius 0.1
    around c(t) = (0.5 + 0.25 cos(6t), 0.5), else 0, at cell centres."""
    nx, ny, nz = dims
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Yc = np.meshgrid(x, y)
    cx, cy = 0.5 + 0.25 * math.cos(6.0 * t), 0.5
    inside = (X - cx) ** 2 + (Yc - cy) ** 2 <= 0.01
    src = np.where(inside, -0.1, 0.0)
    return np.broadcast_to(src, (nz, ny, nx)).ravel().copy()


def diffreact_f(dims, t, u):
    """f(t,u) with M u' + f(t,u) = 0, M = I, for the diffusion-reaction problem
    of Sec. 4.2:
    f_P = -sum_Q a_PQ (u_Q - u_P)/h^2 - u_P (1 - u_P) - src_P(t),
    a_PQ = 1 + (u_P^2 + u_Q^2)/2, zero-flux boundary."""
    h = 1.0 / dims[0]
    f = -u * (1.0 - u) - circle_source(dims, t)
    for _, P, Q in _faces(dims):
        a = 1.0 + 0.5 * (u[P] ** 2 + u[Q] ** 2)
        flux = a * (u[Q] - u[P]) / h**2        # into P
        np.add.at(f, P, -flux)
        np.add.at(f, Q, flux)
    return f


def diffreact_jacobian(dims, t, u):
    """Df(t,u) (CSR) of diffreact_f: the Jacobian of Algorithm 1's simplified
    Newton step (Sec. 2.2), in K's pattern."""
    h = 1.0 / dims[0]
    n = int(np.prod(dims))
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [-(1.0 - 2.0 * u)]
    for _, P, Q in _faces(dims):
        a = 1.0 + 0.5 * (u[P] ** 2 + u[Q] ** 2)
        du = u[Q] - u[P]
        # f_P contains -a (u_Q - u_P)/h^2; f_Q contains +a (u_Q - u_P)/h^2
        dP_uP = (a - u[P] * du) / h**2
        dP_uQ = -(a + u[Q] * du) / h**2
        dQ_uQ = (a + u[Q] * du) / h**2
        dQ_uP = -(a - u[P] * du) / h**2
        rows += [P, P, Q, Q]
        cols += [P, Q, Q, P]
        vals += [dP_uP, dP_uQ, dQ_uQ, dQ_uP]
    return _csr(rows, cols, vals, n)


# --------------------------------------------------------------------------
# Richards' equation with van Genuchten-Mualem (Eq. RelationshipsThetaK)
# --------------------------------------------------------------------------
class VanGenuchten:
    """theta(psi) = theta_R + (theta_S - theta_R) (1 + (-alpha psi)^n)^(-(n-1)/n)
    for psi <= 0, theta_S for psi > 0; relative permeability
    kr = (theta/theta_S)^(1/2) [1 - (1 - (theta/theta_S)^(n/(n-1)))^((n-1)/n)]^2
    (Eq. RelationshipsThetaK with K = K_S kr)."""

    def __init__(self, alpha, n, theta_r, theta_s):
        self.alpha, self.n, self.tr, self.ts = alpha, n, theta_r, theta_s
        self.m = (n - 1.0) / n

    def theta(self, psi):
        psi = np.asarray(psi, dtype=np.float64)
        neg = np.minimum(psi, 0.0)
        u = (-self.alpha * neg) ** self.n
        th = self.tr + (self.ts - self.tr) * (1.0 + u) ** (-self.m)
        return np.where(psi > 0.0, self.ts, th)

    def dtheta(self, psi):
        psi = np.asarray(psi, dtype=np.float64)
        neg = np.minimum(psi, 0.0)
        a, n, m = self.alpha, self.n, self.m
        x = -a * neg
        d = (self.ts - self.tr) * m * n * a * x ** (n - 1.0) * (1.0 + x ** n) ** (-m - 1.0)
        return np.where(psi >= 0.0, 0.0, d)

    def lipschitz(self, samples=200001):
        """sup_psi theta'(psi), the L of the L-scheme (Sec. 4.3): the maximum of
        dtheta over a log-spaced scan of alpha |psi| in [1e-4, 1e4], refined by
        golden-section search around the best sample."""
        x = np.logspace(-4.0, 4.0, samples)
        d = self.dtheta(-x / self.alpha)
        i = int(np.argmax(d))
        lo, hi = x[max(i - 1, 0)], x[min(i + 1, samples - 1)]
        g = (np.sqrt(5.0) - 1.0) / 2.0
        f = lambda t: float(self.dtheta(np.array([-t / self.alpha]))[0])
        for _ in range(200):
            a, b = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(a) >= f(b):
                hi = b
            else:
                lo = a
        return max(f(0.5 * (lo + hi)), float(d[i]))

    def kr(self, psi):
        x = self.theta(psi) / self.ts
        w = 1.0 - x ** (1.0 / self.m)
        w = np.maximum(w, 0.0)
        return np.sqrt(x) * (1.0 - w ** self.m) ** 2

    def dkr(self, psi):
        """d kr / d psi = (d kr / d theta) theta'(psi); zero where psi >= 0 or
        where 1 - x^(1/m) < 1e-12 (saturated limit)."""
        psi = np.asarray(psi, dtype=np.float64)
        x = self.theta(psi) / self.ts
        m = self.m
        w = 1.0 - x ** (1.0 / m)
        ok = (psi < 0.0) & (w > 1e-12)
        ws = np.where(ok, w, 1.0)
        bracket = 1.0 - ws ** m
        dk_dx = 0.5 / np.sqrt(x) * bracket ** 2 + \
            np.sqrt(x) * 2.0 * bracket * ws ** (m - 1.0) * x ** (1.0 / m - 1.0)
        return np.where(ok, dk_dx / self.ts * self.dtheta(psi), 0.0)


def richards_dirichlet_head(t, dt_D):
    """Top-patch Dirichlet pressure head: -2 + 2.2 t/dt_D for t <= dt_D, then
    0.2 (the ramp of the trench boundary in Sec. 4.3)."""
    return -2.0 + 2.2 * t / dt_D if t <= dt_D else 0.2


def richards_cells(dims):
    """Cell-centre heights z and the top-patch mask (top layer, x < 1/2,
    y < 1/2): the inflow boundary of the trench problem of Sec. 4.3."""
    nx, ny, nz = dims
    h = 1.0 / nx
    idx = grid_index(dims)
    z = np.broadcast_to(((np.arange(nz) + 0.5) * h)[:, None, None], (nz, ny, nx)).ravel().copy()
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    top = np.zeros((nz, ny, nx), dtype=bool)
    top[-1] = (x[None, :] < 0.5) & (y[:, None] < 0.5)
    return z, idx[top].ravel()


def _upwind_is_Q(HP, HQ, P, Q):
    """True where the upwind cell of face (P,Q) is Q: head of Q higher, or a
    tie and Q has the lower index."""
    return (HQ > HP) | ((HQ == HP) & (Q < P))


def richards_f(dims, t, psi, Ks, vg: VanGenuchten, dt_D):
    """f(t,psi) with d/dt theta(psi) + f = 0 (Richards' equation, Sec. 4.3,
    Eq. RelationshipsThetaK for theta and K):
    f_P = -sum_Q K_PQ (H_Q - H_P)/h^2 - [top patch] 2 K_S,P kr_up (H_D - H_P)/h^2,
    H = psi + z, K_PQ = harmonic(K_S) kr(upwind)."""
    h = 1.0 / dims[0]
    Ksr = np.asarray(Ks, dtype=np.float64).ravel()
    z, top = richards_cells(dims)
    H = psi + z
    kr = vg.kr(psi)
    f = np.zeros_like(psi)
    for _, P, Q in _faces(dims):
        kf = 2.0 * Ksr[P] * Ksr[Q] / (Ksr[P] + Ksr[Q])
        up = _upwind_is_Q(H[P], H[Q], P, Q)
        K = kf * np.where(up, kr[Q], kr[P])
        flux = K * (H[Q] - H[P]) / h**2
        np.add.at(f, P, -flux)
        np.add.at(f, Q, flux)
    psiD = richards_dirichlet_head(t, dt_D)
    HD = psiD + 1.0
    krD = vg.kr(np.array([psiD]))[0]
    P = top
    up = HD > H[P]
    K = Ksr[P] * np.where(up, krD, kr[P])
    f[P] -= 2.0 * K * (HD - H[P]) / h**2
    return f


def richards_jacobian(dims, t, psi, Ks, vg: VanGenuchten, dt_D, frozen=False):
    """Df(t,psi) (CSR) of richards_f. frozen=True drops the derivative of kr:
    the matrix of the linear flux operator with the conductivities fixed at
    psi (the conductivity part of the L-scheme of Sec. 4.3)."""
    h = 1.0 / dims[0]
    n = int(np.prod(dims))
    Ksr = np.asarray(Ks, dtype=np.float64).ravel()
    z, top = richards_cells(dims)
    H = psi + z
    kr = vg.kr(psi)
    dkr = np.zeros_like(psi) if frozen else vg.dkr(psi)
    rows, cols, vals = [], [], []
    for _, P, Q in _faces(dims):
        kf = 2.0 * Ksr[P] * Ksr[Q] / (Ksr[P] + Ksr[Q])
        up = _upwind_is_Q(H[P], H[Q], P, Q)
        K = kf * np.where(up, kr[Q], kr[P])
        dK_dQ = np.where(up, kf * dkr[Q], 0.0)
        dK_dP = np.where(up, 0.0, kf * dkr[P])
        dH = H[Q] - H[P]
        # f_P = -K dH / h^2 ; f_Q = +K dH / h^2
        dP_P = (K - dK_dP * dH) / h**2
        dP_Q = -(K + dK_dQ * dH) / h**2
        dQ_Q = (K + dK_dQ * dH) / h**2
        dQ_P = -(K - dK_dP * dH) / h**2
        rows += [P, P, Q, Q]
        cols += [P, Q, Q, P]
        vals += [dP_P, dP_Q, dQ_Q, dQ_P]
    psiD = richards_dirichlet_head(t, dt_D)
    HD = psiD + 1.0
    krD = vg.kr(np.array([psiD]))[0]
    P = top
    up = HD > H[P]
    K = Ksr[P] * np.where(up, krD, kr[P])
    dK = np.where(up, 0.0, Ksr[P] * dkr[P])   # zero when frozen
    rows.append(P)
    cols.append(P)
    vals.append(2.0 * (K - dK * (HD - H[P])) / h**2)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(np.zeros(n))
    return _csr(rows, cols, vals, n)
