"""Pins of oracle.coupling against the paper's printed matrices and against
independent derivations (CPU only)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupling, fv, slab

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals, mats, cur = {}, {}, None
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("theta", "tau", "s"):
                vals[parts[0]] = float(parts[1])
            elif parts[0].isalpha() or parts[0] in ("A1", "A2"):
                cur = parts[0]
                mats[cur] = []
            else:
                mats[cur].append([float(x) for x in parts])
    return vals, {k: np.array(v) for k, v in mats.items()}


def test_theta_example_matches_printed_matrices():
    """Example ex:time-stepping-matrices (printed closed form, hand-written)."""
    v, m = _read_golden("theta_example_s4.txt")
    A, b, c = coupling.theta_method(v["theta"])
    A1, A2, e = coupling.multistep_matrices(A, int(v["s"]), v["tau"], eliminate_first=True)
    np.testing.assert_allclose(A1, m["A1"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(A2, m["A2"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(e, [1.0 - v["theta"]])
    A1c, A2c = coupling.theta_example_matrices(v["theta"], int(v["s"]), v["tau"])
    np.testing.assert_allclose(A1c, m["A1"], atol=1e-15)
    np.testing.assert_allclose(A2c, m["A2"], atol=1e-15)


def test_stiffly_accurate_tableaux():
    for A, b, c in (coupling.implicit_euler(), coupling.theta_method(0.5), coupling.sdirk2()):
        assert coupling.is_stiffly_accurate(A, b)
        np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-15)   # row-sum condition


def _small_problem(seed=0, n=4):
    dims = (n, n, 1)
    rng = np.random.default_rng(seed)
    D = np.exp(rng.standard_normal((1, n, n)))
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
    Mdiag = 1.0 + rng.random(n * n)
    return K, Mdiag, rng


def test_theta_one_step_form():
    """Eliminated theta-method, s = 1, equals the printed one-step form
    (M/tau + theta K) y^{n+1} = theta b^{n+1} + M y^n / tau + (1-theta)(b^n - K y^n)."""
    K, Md, rng = _small_problem(1)
    n = K.shape[0]
    th, tau = 0.3, 0.05
    yn, bn, bn1 = rng.standard_normal((3, n))
    A, _, _ = coupling.theta_method(th)
    A1, A2, e = coupling.multistep_matrices(A, 1, tau, eliminate_first=True)
    B0 = (Md * yn / tau + e[0] * (bn - K @ yn))[:, None]
    Y = slab.solve_all_at_once_dense(K, Md, A1, A2, bn1[:, None], B0)
    direct = np.linalg.solve(np.diag(Md) / tau + th * K.toarray(),
                             th * bn1 + Md * yn / tau + (1 - th) * (bn - K @ yn))
    np.testing.assert_allclose(Y[:, 0], direct, rtol=1e-12, atol=1e-12)
    B0ex = coupling.theta_example_B0(th, tau, Md, K, yn, bn, 1)
    np.testing.assert_allclose(B0, B0ex, rtol=1e-14, atol=1e-14)


def test_elimination_keeps_the_solution():
    """Solving the 2-stage theta system with the explicit stage kept gives the
    same y^{n+1} as the eliminated system (Sec. 2.1 elimination)."""
    K, Md, rng = _small_problem(2)
    n = K.shape[0]
    th, tau = 0.6, 0.1
    yn, bn, bn1 = rng.standard_normal((3, n))
    A, _, _ = coupling.theta_method(th)
    A1, A2 = coupling.single_step_matrices(A, tau)
    B = np.column_stack([bn, bn1])
    B0 = np.column_stack([Md * yn / tau, Md * yn / tau])
    Yfull = slab.solve_all_at_once_dense(K, Md, A1, A2, B, B0)
    np.testing.assert_allclose(Yfull[:, 0], yn, rtol=1e-12, atol=1e-12)
    A1e, A2e, e = coupling.multistep_matrices(A, 1, tau, eliminate_first=True)
    B0e = (Md * yn / tau + e[0] * (bn - K @ yn))[:, None]
    Ye = slab.solve_all_at_once_dense(K, Md, A1e, A2e, bn1[:, None], B0e)
    np.testing.assert_allclose(Ye[:, 0], Yfull[:, 1], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("tab", ["ie", "sdirk2"])
def test_window_at_step_boundary_equals_multistep(tab):
    A, b, c = coupling.implicit_euler() if tab == "ie" else coupling.sdirk2()
    m = A.shape[0]
    tau = 0.1
    for steps in (1, 2, 3):
        A1, A2, _ = coupling.multistep_matrices(A, steps, tau)
        W1, W2, terms, times = coupling.window_matrices(A, c, tau, 2 * m, steps * m)
        np.testing.assert_allclose(W1, A1, atol=1e-15)
        np.testing.assert_allclose(W2, A2, atol=1e-15)
        # only the first step's stages see the known y^n (mass term)
        assert {t[0] for t in terms if t[1] == "mass"} == set(range(m))
        assert all(t[1] == "mass" for t in terms)


def test_window_mid_step_sdirk2():
    """Window starting at stage (n,2): column 0 gets B0 = M y^n / tau - a21 f(n,1),
    column 1 = (n+1, 1) couples to column 0 through A1[1,0] = -1/tau."""
    A, b, c = coupling.sdirk2()
    tau = 0.2
    g = A[0, 0]
    W1, W2, terms, times = coupling.window_matrices(A, c, tau, 3, 2)   # stage (1,2)
    np.testing.assert_allclose(W1, [[1 / tau, 0], [-1 / tau, 1 / tau]], atol=1e-15)
    np.testing.assert_allclose(W2, [[g, 0], [0, g]], atol=1e-15)
    assert sorted(terms) == sorted([(0, "mass", 1, 1 / tau), (0, "f", 2, -(1 - g))])
    np.testing.assert_allclose(times, [2 * tau, (2 + g) * tau])


def test_stage_map_and_shift():
    assert [coupling.stage_of(g, 3) for g in range(7)] == \
        [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 1)]
    Y = np.arange(12.0).reshape(3, 4)
    S = coupling.shift(Y)
    np.testing.assert_array_equal(S[:, :3], Y[:, 1:])
    np.testing.assert_array_equal(S[:, 3], Y[:, 3])


def test_splitting_parts():
    A, _, _ = coupling.theta_method(0.3)
    A1, A2, _ = coupling.multistep_matrices(A, 5, 0.5, eliminate_first=True)
    alpha, beta, O1, O2 = coupling.splitting(A1, A2)
    assert alpha == 2.0 and beta == 0.3
    # after elimination the split-off parts are strictly lower triangular
    assert np.allclose(np.triu(O1), 0) and np.allclose(np.triu(O2), 0)
