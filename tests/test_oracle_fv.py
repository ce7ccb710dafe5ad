"""Pins of oracle.fv: convergence orders, conservation, symmetry, pattern
sizes, finite-difference Jacobians, van Genuchten limits (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from oracle import fv


def test_pattern_nnz_of_the_workload_grids():
    assert fv.pattern((64, 64, 1)).nnz == 20224
    assert fv.pattern((16, 16, 16)).nnz == 7 * 16**3 - 6 * 16**2
    K = fv.convdiff_matrix((8, 8, 8), np.ones((8, 8, 8)), (1.0, 0.5, 0.0))
    assert K.nnz == 7 * 512 - 6 * 64


def test_diffusion_second_order_mms():
    """-Laplace u = f on [0,1]^2, u = sin(pi x) sin(pi y): error O(h^2)."""
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        X, Y = np.meshgrid(x, x)
        u = (np.sin(np.pi * X) * np.sin(np.pi * Y)).ravel()
        f = 2 * np.pi**2 * u
        K = fv.convdiff_matrix((n, n, 1), np.ones((1, n, n)), (0.0, 0.0, 0.0))
        uh = spsolve(K.tocsc(), f)
        errs.append(np.max(np.abs(uh - u)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), rates


def test_upwind_first_order_mms():
    """-u'' + v u' with v = 20 in 1-D strips: error O(h) (upwind)."""
    errs = []
    v = 20.0
    for n in (64, 128, 256):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        u = np.sin(np.pi * x)
        f = np.pi**2 * np.sin(np.pi * x) + v * np.pi * np.cos(np.pi * x)
        K = fv.convdiff_matrix((n, 1, 1), np.ones((1, 1, n)), (v, 0.0, 0.0))
        uh = spsolve(K.tocsc(), f)
        errs.append(np.max(np.abs(uh - u)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 0.8) and np.all(rates < 1.5), rates


def test_conservation_and_symmetry():
    rng = np.random.default_rng(0)
    dims = (6, 5, 4)
    D = np.exp(rng.standard_normal(dims[::-1]))
    K0 = fv.convdiff_matrix(dims, D, (0.0, 0.0, 0.0))
    assert abs(K0 - K0.T).max() < 1e-12
    K = fv.convdiff_matrix(dims, D, (1.0, -0.5, 0.25))
    Kb = fv.convdiff_matrix(dims, D, (0.0, 0.0, 0.0))
    # interior faces conserve: column sums equal the boundary (ghost + outflow) terms only
    colsum = np.asarray(K.sum(axis=0)).ravel() - np.asarray(Kb.sum(axis=0)).ravel()
    h = 1.0 / dims[0]
    idx = fv.grid_index(dims)
    expect = np.zeros(K.shape[0])
    expect[idx[:, :, -1].ravel()] += 1.0 / h       # vx > 0 leaves at x = 1
    expect[idx[:, 0, :].ravel()] += 0.5 / h        # vy < 0 leaves at y = 0
    expect[idx[-1, :, :].ravel()] += 0.25 / h      # vz > 0 leaves at z = 1
    np.testing.assert_allclose(colsum, expect, rtol=1e-12, atol=1e-9)


def _fd_jacobian(fun, y, eps=1e-6):
    n = len(y)
    Jd = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        Jd[:, j] = (fun(y + e) - fun(y - e)) / (2 * eps)
    return Jd


def test_diffreact_jacobian_matches_finite_differences():
    dims = (5, 4, 1)
    rng = np.random.default_rng(1)
    u = rng.uniform(0.1, 0.9, 20)
    t = 0.3
    J = fv.diffreact_jacobian(dims, t, u).toarray()
    Jd = _fd_jacobian(lambda v: fv.diffreact_f(dims, t, v), u)
    np.testing.assert_allclose(J, Jd, rtol=1e-6, atol=1e-5)


def test_diffreact_conservation():
    """Without reaction and source the fluxes sum to zero (Neumann)."""
    dims = (7, 6, 1)
    rng = np.random.default_rng(2)
    u = rng.uniform(0, 1, 42)
    f = fv.diffreact_f(dims, 0.0, u) + u * (1 - u) + fv.circle_source(dims, 0.0)
    assert abs(f.sum()) < 1e-9


def test_van_genuchten_limits():
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    assert vg.theta(np.array([0.0]))[0] == pytest.approx(0.4)
    assert vg.theta(np.array([1.0]))[0] == pytest.approx(0.4)
    assert vg.theta(np.array([-1e8]))[0] == pytest.approx(0.05, abs=1e-6)
    assert vg.kr(np.array([0.0]))[0] == pytest.approx(1.0)
    psi = -np.logspace(-3, 2, 200)[::-1]
    th = vg.theta(psi)
    assert np.all(np.diff(th) > 0)                  # monotone in psi
    kr = vg.kr(psi)
    assert np.all(np.diff(kr) >= -1e-15)
    # closed form for n = 2: theta = tr + (ts-tr)/sqrt(1 + psi^2)
    np.testing.assert_allclose(th, 0.05 + 0.35 / np.sqrt(1 + psi**2), rtol=1e-13)
    d = (vg.theta(psi + 1e-7) - vg.theta(psi - 1e-7)) / 2e-7
    np.testing.assert_allclose(vg.dtheta(psi), d, rtol=1e-5, atol=1e-9)
    dk = (vg.kr(psi + 1e-7) - vg.kr(psi - 1e-7)) / 2e-7
    sel = psi < -1e-2
    np.testing.assert_allclose(vg.dkr(psi)[sel], dk[sel], rtol=1e-4, atol=1e-8)


def test_van_genuchten_kr_closed_form():
    """kr of Eq. RelationshipsThetaK, K/K_S = x^(1/2) [1 - (1 - x^(n/(n-1)))^((n-1)/n)]^2
    with x = theta/theta_S, against values worked out independently:
     * n = 2 (exponents 2 and 1/2): theta = tr + (ts - tr)/sqrt(1 + psi^2) and
       kr = sqrt(x) (1 - sqrt(1 - x^2))^2, written out here;
     * the same and an n = 3 case (exponents 3/2 and 2/3) evaluated in exact
       rational arithmetic beforehand (25 digits, literals below).
    Swapping the two exponents keeps kr(0) = 1 and monotonicity but changes
    every interior value (at n = 2, psi = -1: 0.830 instead of 0.0948)."""
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    psi = np.array([-0.5, -1.0, -3.0])
    x = (0.05 + 0.35 / np.sqrt(1.0 + psi ** 2)) / 0.4
    np.testing.assert_allclose(vg.kr(psi), np.sqrt(x) * (1.0 - np.sqrt(1.0 - x ** 2)) ** 2,
                               rtol=1e-12)
    exact_n2 = [0.3207240617325334723442305, 0.09477410205668127813004689,
                0.004496424850521366630713021]
    np.testing.assert_allclose(vg.kr(psi), exact_n2, rtol=1e-12)
    # n = 3, alpha = 1, psi = -1: theta = tr + (ts - tr) 2^(-2/3)
    vg3 = fv.VanGenuchten(1.0, 3.0, 0.05, 0.4)
    assert vg3.theta(np.array([-1.0]))[0] / 0.4 == pytest.approx(0.6762154593290070095856546,
                                                                 rel=1e-13)
    assert vg3.kr(np.array([-1.0]))[0] == pytest.approx(0.1437211805412071599323933, rel=1e-12)
    # n = 3, alpha = 2, psi = -0.75 (alpha |psi| = 3/2)
    vg3b = fv.VanGenuchten(2.0, 3.0, 0.05, 0.4)
    assert vg3b.kr(np.array([-0.75]))[0] == pytest.approx(0.03097319362505719719299625,
                                                           rel=1e-12)


def test_richards_jacobian_matches_finite_differences():
    dims = (4, 4, 4)
    rng = np.random.default_rng(3)
    Ks = np.exp(rng.standard_normal(dims[::-1]))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    psi = -z - 0.3 + 0.2 * rng.standard_normal(64)
    t = 0.01
    J = fv.richards_jacobian(dims, t, psi, Ks, vg, 1 / 16).toarray()
    Jd = _fd_jacobian(lambda p: fv.richards_f(dims, t, p, Ks, vg, 1 / 16), psi, 1e-7)
    np.testing.assert_allclose(J, Jd, rtol=1e-5, atol=1e-4)


def test_richards_hydrostatic_is_steady_without_boundary_flux():
    """psi = -z (H constant) gives no interior flux; only the top patch acts."""
    dims = (6, 6, 6)
    Ks = np.ones(dims[::-1])
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, top = fv.richards_cells(dims)
    f = fv.richards_f(dims, 0.0, -z, Ks, vg, 1 / 16)
    mask = np.ones(216, dtype=bool)
    mask[top] = False
    np.testing.assert_allclose(f[mask], 0.0, atol=1e-12)
    assert np.all(f[top] > 0.0)      # psi_D = -2 below hydrostatic: water leaves


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_vg_lipschitz_matches_paper_silt_loam():
    """Sec. 4.3 chooses L as the Lipschitz constant of Theta for the silt loam
    of its parameter table and prints L = 4.501e-2 (golden file
    silt_loam_lscheme.txt)."""
    g = _golden("silt_loam_lscheme.txt")
    vg = fv.VanGenuchten(g["alpha"], g["n"], g["theta_R"], g["theta_S"])
    assert abs(vg.lipschitz() - g["L"]) < 0.0005e-2


def test_vg_lipschitz_is_the_supremum():
    """L bounds theta' everywhere and is attained, at alpha |psi| = m^(1/n)
    (the stationary point of theta')."""
    for a, n, tr, ts in [(1.0, 2.0, 0.05, 0.4), (0.423, 2.06, 0.131, 0.396), (3.0, 1.4, 0.0, 0.5)]:
        vg = fv.VanGenuchten(a, n, tr, ts)
        L = vg.lipschitz()
        psi = -np.logspace(-6, 6, 20001)
        assert np.all(vg.dtheta(psi) <= L * (1 + 1e-12))
        m = 1.0 - 1.0 / n
        x = m ** (1.0 / n)
        np.testing.assert_allclose(vg.dtheta(np.array([-x / a]))[0], L, rtol=1e-12)
        # theta is L-Lipschitz: |theta(p) - theta(q)| <= L |p - q|
        p, q = psi[:-1], psi[1:]
        assert np.all(np.abs(vg.theta(p) - vg.theta(q)) <= L * np.abs(p - q) * (1 + 1e-9))


def test_richards_frozen_jacobian():
    """The L-scheme's conductivity part: symmetric (one conductivity per face,
    harmonic K_S), equal to the full Jacobian where kr is constant (saturated
    soil, psi > 0), and the exact derivative of f with kr held at psi0."""
    dims = (5, 4, 3)
    n = 60
    rng = np.random.default_rng(3)
    Ks = np.exp(rng.standard_normal(dims[::-1]))
    vg = fv.VanGenuchten(1.0, 2.0, 0.05, 0.4)
    z, _ = fv.richards_cells(dims)
    psi = -z - 0.3 + 0.2 * rng.random(n)
    A = fv.richards_jacobian(dims, 0.02, psi, Ks, vg, 1 / 16, frozen=True).toarray()
    np.testing.assert_allclose(A, A.T, rtol=1e-13, atol=1e-12)
    wet = 0.5 + rng.random(n)
    np.testing.assert_allclose(
        fv.richards_jacobian(dims, 0.02, wet, Ks, vg, 1 / 16, frozen=True).toarray(),
        fv.richards_jacobian(dims, 0.02, wet, Ks, vg, 1 / 16).toarray(), rtol=1e-13, atol=1e-12)
    # with kr frozen f is affine in psi as long as no face changes its upwind
    # side: f(psi0 + d) - f_frozen... checked on a small perturbation
    d = 1e-7 * rng.standard_normal(n)
    kr0 = vg.kr(psi)

    class Frozen(fv.VanGenuchten):
        def kr(self, p):
            return kr0
    f0 = fv.richards_f(dims, 0.02, psi, Ks, Frozen(1.0, 2.0, 0.05, 0.4), 1 / 16)
    f1 = fv.richards_f(dims, 0.02, psi + d, Ks, Frozen(1.0, 2.0, 0.05, 0.4), 1 / 16)
    np.testing.assert_allclose(f1 - f0, A @ d, rtol=1e-5, atol=1e-12)
