"""GPU parity of the building-block kernels against the oracle (float64
definition) through the C ABI. Sizes span several SELL slices / CTAs and a
ragged tail (N not a multiple of 32)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import coupling, fv, krylov, slab

pytestmark = pytest.mark.gpu

DIMS = [(13, 11, 7), (64, 64, 1), (5, 3, 1)]
SS = [1, 2, 3, 4, 5, 8, 13, 16]


def _dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda",
                        dtype=dtype or torch.float64)


def _problem(dims, seed=0, v=(1.0, -0.5, 0.25)):
    n = int(np.prod(dims))
    D = np.exp(synth.normal(seed, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, v if dims[2] > 1 else (v[0], v[1], 0.0))
    return D, K, n


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("s", SS)
def test_apply_coupled_matches_oracle(P, ctx, dims, s):
    import torch
    D, K, n = _problem(dims, 1)
    v = (1.0, -0.5, 0.25) if dims[2] > 1 else (1.0, -0.5, 0.0)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), v)
    try:
        rng = np.random.default_rng(s)
        A1 = rng.standard_normal((s, s))
        A2 = rng.standard_normal((s, s))
        A1[0, 0] = 3.0
        A1[np.abs(A1) < 0.3] = 0.0          # exercise the zero-skipping branches
        P.pint_set_coupling(ctx, op, A1, A2)
        Y, B, B0 = (synth.uniform(10 + i, n * s).reshape(n, s) for i in range(3))
        R = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_apply_coupled(ctx, op, _dev(Y), _dev(B), _dev(B0), R)
        ref = slab.coupled_residual(K, np.ones(n), A1, A2, Y, B, B0)
        scale = np.abs(K).max() * np.abs(A2).sum(axis=1).max() * 10
        np.testing.assert_allclose(R.cpu().numpy(), ref, rtol=0, atol=1e-13 * scale)
        P.pint_apply_coupled(ctx, op, _dev(Y), None, None, R)
        ref = slab.coupled_residual(K, np.ones(n), A1, A2, Y)
        np.testing.assert_allclose(R.cpu().numpy(), ref, rtol=0, atol=1e-13 * scale)
    finally:
        P.pint_operator_destroy(op)


def test_operator_assemble_csr_with_mass(P, ctx):
    """User CSR (host and device) with a diagonal mass matrix."""
    import torch
    D, K, n = _problem((9, 7, 5), 2)
    rng = np.random.default_rng(0)
    M = 0.5 + rng.random(n)
    s = 4
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, 0.01)
    Y = rng.standard_normal((n, s))
    ref = slab.coupled_residual(K, M, A1, A2, Y)
    for dev in (False, True):
        args = [K.indptr.astype(np.int32), K.indices.astype(np.int32), K.data, M]
        if dev:
            args = [torch.tensor(a, device="cuda") for a in args]
        op = P.pint_operator_assemble(ctx, n, *args)
        P.pint_set_coupling(ctx, op, A1, A2)
        R = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_apply_coupled(ctx, op, _dev(Y), None, None, R)
        np.testing.assert_allclose(R.cpu().numpy(), ref, rtol=1e-14, atol=1e-9)
        assert P.pint_operator_nnz(op) == K.nnz
        P.pint_operator_destroy(op)


def test_operator_assemble_rejects_bad_csr(P, ctx):
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 0], dtype=np.int32)       # no diagonal entries
    with pytest.raises(P.PintError):
        P.pint_operator_assemble(ctx, 2, rp, ci, np.ones(2))


@pytest.mark.parametrize("path", ["stencil", "csr"])
@pytest.mark.parametrize("dims", [(13, 11, 7), (40, 33, 1), (37, 1, 1)])
@pytest.mark.parametrize("s", [1, 3, 8, 16])
def test_inner_apply_and_jacobi(P, ctx, s, dims, path):
    """J X and the Jacobi step against the oracle's CSR product, for grid
    operators (stencil-form SpMM) and the same matrix assembled as plain CSR
    (SELL-32 SpMM)."""
    import torch
    D, K, n = _problem(dims, 3)
    v = (1.0, -0.5, 0.25) if dims[2] > 1 else (1.0, -0.5, 0.0)
    if dims[1] == 1:
        v = (1.0, 0.0, 0.0)
    K = fv.convdiff_matrix(dims, D, v)
    if path == "stencil":
        op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), v)
    else:
        Kc = K.tocsr()
        Kc.sort_indices()
        op = P.pint_operator_assemble(ctx, n, Kc.indptr.astype(np.int32),
                                      Kc.indices.astype(np.int32), Kc.data)
    try:
        A, _, _ = coupling.sdirk2()
        tau = 0.02
        A1 = np.eye(s) / tau
        A2 = np.eye(s) * A[0, 0]
        P.pint_set_coupling(ctx, op, A1, A2)
        X = synth.uniform(5, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_inner_apply(ctx, op, _dev(X), Z)
        J = sp.identity(n) / tau + A[0, 0] * K
        np.testing.assert_allclose(Z.cpu().numpy(), J @ X, rtol=1e-13, atol=1e-10)
        P.pint_precond_apply(ctx, op, P.PINT_PC_JACOBI, _dev(X), Z)
        np.testing.assert_allclose(Z.cpu().numpy(), krylov.jacobi(J.tocsr())(X), rtol=1e-15)
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("path", ["stencil", "csr"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("s", [1, 4, 8, 16])
def test_inner_apply_low_precision(P, ctx, s, prec, path):
    """Z = J X with the float32 / bfloat16 copies of J (float32 vectors and
    accumulation) against the float64 CSR product. Per entry the error is a
    few roundings of the matrix values (2^-24 / 2^-9 relative) and of the
    float32 products, relative to sum_j |J_ij| |X_j|."""
    import torch
    dims = (21, 13, 9)
    D, K, n = _problem(dims, 5)
    if path == "stencil":
        op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, -0.5, 0.25))
    else:
        Kc = K.tocsr()
        Kc.sort_indices()
        op = P.pint_operator_assemble(ctx, n, Kc.indptr.astype(np.int32),
                                      Kc.indices.astype(np.int32), Kc.data)
    try:
        tau = 0.01
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        X = synth.uniform(9, n * s).reshape(n, s).astype(np.float32)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float32)
        code = P.PINT_FP32 if prec == "fp32" else P.PINT_BF16
        P.pint_inner_apply_lowp(ctx, op, code, torch.tensor(X, device="cuda"), Z)
        torch.cuda.synchronize()
        J = (sp.identity(n) / tau + K).tocsr()
        ref = J @ X.astype(np.float64)
        scale = abs(J) @ np.abs(X.astype(np.float64))
        rel = 16 * 2.0 ** -24 if prec == "fp32" else 2.0 ** -8
        assert np.all(np.abs(Z.cpu().numpy() - ref) <= rel * scale + 1e-30)
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("dims", [(13, 11, 7), (40, 33, 1)])
@pytest.mark.parametrize("s", [1, 3, 8, 16])
def test_ilu0_apply_matches_oracle(P, ctx, dims, s):
    import torch
    D, K, n = _problem(dims, 4)
    v = (1.0, -0.5, 0.25) if dims[2] > 1 else (1.0, -0.5, 0.0)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), v)
    try:
        tau = 1e-3
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        J = sp.csr_matrix(sp.identity(n) / tau + K)
        J.sort_indices()
        X = synth.uniform(6, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_precond_apply(ctx, op, P.PINT_PC_ILU0, _dev(X), Z)
        ref = krylov.ilu0_apply(*krylov.ilu0(J))(X)
        np.testing.assert_allclose(Z.cpu().numpy(), ref, rtol=1e-11, atol=1e-14)
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("n", [4099, 65536])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s,nb", [(1, 1), (1, 31), (3, 7), (4, 31), (8, 12), (16, 1), (16, 31)])
def test_gram_update_colnorms(P, ctx, prec, s, nb, n):
    """n = 4099: plain-load Gram kernel; n = 65536 (a multiple of 64): the
    bulk-copy (TMA) pipeline with several tiles per CTA."""
    import torch
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
    V = synth.uniform(7, nb * n * s).reshape(nb, n, s)
    W = synth.uniform(8, n * s).reshape(n, s)
    if prec == "fp32":
        V = V.astype(np.float32).astype(np.float64)
        W = W.astype(np.float32).astype(np.float64)
    Vd, Wd = _dev(V, dt), _dev(W, dt)
    H = torch.empty(nb * s, s, device="cuda", dtype=torch.float64)
    P.pint_block_gram(ctx, code, n, s, nb, Vd, Wd, H)
    Vm = np.concatenate([V[b] for b in range(nb)], axis=1)      # n x (nb s)
    ref = Vm.T @ W
    tol = 1e-12 if prec == "fp64" else 2e-5
    np.testing.assert_allclose(H.cpu().numpy(), ref, rtol=0, atol=tol * np.sqrt(n))
    Hh = synth.uniform(9, nb * s * s).reshape(nb * s, s) * 0.1
    P.pint_block_update(ctx, code, n, s, nb, Vd, _dev(Hh), Wd)
    ref = W - Vm @ Hh
    tol = 1e-13 if prec == "fp64" else 1e-5
    np.testing.assert_allclose(Wd.double().cpu().numpy(), ref, rtol=0, atol=tol * nb * s)
    nrm = P.pint_colnorms(ctx, code, n, s, Wd)
    np.testing.assert_allclose(nrm, np.linalg.norm(Wd.double().cpu().numpy(), axis=0),
                               rtol=1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec,s,nb", [("fp32", 1, 300), ("fp64", 2, 300), ("fp32", 1, 700)])
def test_gram_many_blocks_bulk_pipeline(P, ctx, prec, s, nb):
    """More basis blocks than the Gram CTA has threads (nb + 1 > 256): every
    block must still be copied into each stage of the bulk-copy ring (n a
    multiple of 64 takes that pipeline). Checked against V^T W in float64."""
    import torch
    n = 65536
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
    Vd = torch.tensor(synth.uniform(17, nb * n * s).reshape(nb, n, s), device="cuda", dtype=dt)
    Wd = torch.tensor(synth.uniform(18, n * s).reshape(n, s), device="cuda", dtype=dt)
    H = torch.full((nb * s, s), float("nan"), device="cuda", dtype=torch.float64)
    P.pint_block_gram(ctx, code, n, s, nb, Vd, Wd, H)
    Vm = Vd.double().cpu().numpy().transpose(0, 2, 1).reshape(nb * s, n)
    Wm = Wd.double().cpu().numpy()
    scale = np.abs(Vm) @ np.abs(Wm)
    err = np.abs(H.cpu().numpy() - Vm @ Wm)
    assert np.all(err <= (1e-13 if prec == "fp64" else 1e-5) * scale)


@pytest.mark.parametrize("s", [1, 2, 5, 8, 16])
def test_cholqr2_matches_oracle(P, ctx, s):
    import torch
    n = 2053
    W = synth.uniform(3, n * s).reshape(n, s) @ np.diag(np.logspace(0, 3, s))
    Wd = _dev(W)
    R = torch.empty(s, s, device="cuda", dtype=torch.float64)
    P.pint_cholqr2(ctx, P.PINT_FP64, n, s, Wd, R)
    Q = Wd.cpu().numpy()
    Qr, Rr = krylov.cholqr2(W)
    np.testing.assert_allclose(R.cpu().numpy(), Rr, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(Q, Qr, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(s), atol=1e-13)


def test_cholqr2_deflation_no_nan(P, ctx):
    import torch
    n, s = 1000, 4
    W = synth.uniform(4, n * s).reshape(n, s)
    W[:, 2] = W[:, 0]
    W[:, 3] = 0.0
    Wd = _dev(W)
    R = torch.empty(s, s, device="cuda", dtype=torch.float64)
    P.pint_cholqr2(ctx, P.PINT_FP64, n, s, Wd, R)
    Q = Wd.cpu().numpy()
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(R.cpu().numpy()))
    np.testing.assert_allclose(Q[:, 2:], 0.0)
    np.testing.assert_allclose(Q @ R.cpu().numpy(), W, atol=1e-12)


@pytest.mark.parametrize("s", [2, 5, 16])
def test_shift(P, s):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 77
    Y = np.arange(n * s, dtype=np.float64).reshape(n, s)
    Yd = _dev(Y)
    P.pint_shift(Yd, n, s)
    np.testing.assert_array_equal(Yd.cpu().numpy(), coupling.shift(Y))


@pytest.mark.parametrize("s", [1, 4, 16])
def test_ilu0_apply_generic_csr_matches_oracle(P, ctx, s):
    """User CSR operator (no grid shape): the dependency-flag sweep path."""
    import torch
    dims = (11, 9, 6)
    D, K, n = _problem(dims, 8)
    rng = np.random.default_rng(1)
    M = 1.0 + rng.random(n)
    op = P.pint_operator_assemble(ctx, n, K.indptr.astype(np.int32), K.indices.astype(np.int32),
                                  K.data, M)
    try:
        tau = 1e-2
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        J = sp.csr_matrix(sp.diags(M / tau) + K)
        J.sort_indices()
        X = synth.uniform(6, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_precond_apply(ctx, op, P.PINT_PC_ILU0, _dev(X), Z)
        ref = krylov.ilu0_apply(*krylov.ilu0(J))(X)
        np.testing.assert_allclose(Z.cpu().numpy(), ref, rtol=1e-11, atol=1e-14)
    finally:
        P.pint_operator_destroy(op)


def test_ilu0_apply_1d_tiles(P, ctx):
    import torch
    dims = (150, 1, 1)
    D, K, n = _problem(dims, 9, v=(2.0, 0.0, 0.0))
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (2.0, 0.0, 0.0))
    try:
        s = 3
        P.pint_set_coupling(ctx, op, np.eye(s) * 10.0, np.eye(s))
        J = sp.csr_matrix(sp.identity(n) * 10.0 + K)
        X = synth.uniform(7, n * s).reshape(n, s)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_precond_apply(ctx, op, P.PINT_PC_ILU0, _dev(X), Z)
        # tridiagonal: ILU(0) is the exact LU, so the apply is the solve
        np.testing.assert_allclose(J @ Z.cpu().numpy(), X, rtol=1e-12, atol=1e-12)
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("dims", [(24, 16, 32), (16, 48, 16), (40, 24, 17)])
@pytest.mark.parametrize("s", [1, 2, 3, 8])
def test_ilu0_apply_f32_row_sweeps(P, ctx, dims, s):
    """Float32 ILU(0) through the row-of-tiles sweep (several rows and tiles
    per direction, published faces, reciprocal diagonal) against the oracle's
    float64 ILU(0)."""
    import torch
    D, K, n = _problem(dims, 12)
    v = (1.0, -0.5, 0.25)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), v)
    try:
        tau = 1e-3
        P.pint_set_coupling(ctx, op, np.eye(s) / tau, np.eye(s))
        J = sp.csr_matrix(sp.identity(n) / tau + K)
        J.sort_indices()
        X = synth.uniform(13, n * s).reshape(n, s).astype(np.float32)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float32)
        P.pint_ilu0_apply_f32(ctx, op, _dev(X, torch.float32), Z)
        ref = krylov.ilu0_apply(*krylov.ilu0(J))(X.astype(np.float64))
        err = np.linalg.norm(Z.cpu().numpy().astype(np.float64) - ref, axis=0)
        assert np.all(err <= 1e-5 * np.linalg.norm(ref, axis=0)), err / np.linalg.norm(ref, axis=0)
    finally:
        P.pint_operator_destroy(op)
