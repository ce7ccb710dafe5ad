"""Full-size checks in the launch configuration bench.py times: the 128^3
convection-diffusion slab (s = 8 coupled implicit-Euler steps, ILU(0),
float32 inner solve with float64 refinement, and the float64 path), the
512^2 diffusion-reaction and 96^3 Richards pipelines (Algorithm 1).

The oracle cannot solve these systems in seconds, so the checks are outputs
it computes directly at this size (the coupled residual, ILU(0) by
hyperplanes, sampled Gram and update entries) and properties that hold at
any size (the oracle's own float64 residual of the device solution meets the
tolerance; each stored stage satisfies its stage equation)."""
import numpy as np
import pytest

import bench
import synth
from oracle import coupling, fv, krylov, newton, slab

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda",
                        dtype=dtype or torch.float64)


@pytest.fixture(scope="module")
def slab_case(P, ctx):
    case = bench.LinearCase(P, ctx, bench.parse([]))
    w = case.w
    D = synth.diffusion_field(w)
    K = fv.convdiff_matrix(w.dims, D, w.velocity)
    s = case.s
    A1 = (np.eye(s) - np.eye(s, k=-1)) / w.tau
    A2 = np.eye(s)
    yield case, K, A1, A2
    case.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_slab_solution_meets_tolerance_in_oracle_residual(P, slab_case, prec):
    """Eq. (all-at-once system) at 128^3, s = 8: the oracle's float64 CSR
    residual M Y A1^T + (K Y - B) A2^T of the device solution is below
    tol * ||F_k|| in every column (F = B A2^T)."""
    case, K, A1, A2 = slab_case
    case.o.precision = P.PINT_FP32 if prec == "fp32" else P.PINT_FP64
    try:
        st = case.step()
    finally:
        case.o.precision = P.PINT_FP32
    assert st.status == P.PINT_OK
    Y = case.Y.cpu().numpy()
    R = slab.coupled_residual(K, np.ones(case.n), A1, A2, Y, case.B)
    F = slab.rhs_F(A2, case.B)
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(F, axis=0)
    # the device's float64 residual and the oracle's differ only by summation
    # order: O(1e-16 * s) relative to ||F||, far below the 1e-10 target
    assert np.all(rel <= case.w.tol * (1.0 + 1e-3)), rel
    np.testing.assert_allclose(np.array(st.col_relres[:case.s]), rel, rtol=1e-2, atol=1e-14)


def test_coupled_residual_full_size(P, ctx, slab_case):
    """Kernel a2 (Eq. matrix-equation, defect form) at 128^3, s = 8, compared
    entry by entry with the oracle's CSR evaluation."""
    import torch
    case, K, A1, A2 = slab_case
    n, s = case.n, case.s
    Y = synth.uniform(31, n * s).reshape(n, s)
    B0 = synth.uniform(32, n * s).reshape(n, s)
    R = torch.empty(n, s, device="cuda", dtype=torch.float64)
    P.pint_apply_coupled(ctx, case.op, _dev(Y), case.Bd, _dev(B0), R)
    ref = slab.coupled_residual(K, np.ones(n), A1, A2, Y, case.B, B0)
    # terms are O(||K||_inf |Y|); float64 sums of 7 + 2 s terms in another order
    scale = np.asarray(abs(K).sum(axis=1)).ravel() + 2.0 / case.w.tau + 2.0
    np.testing.assert_allclose(R.cpu().numpy(), ref, rtol=0,
                               atol=1e-14 * float(scale.max()) * 16)


def _ilu_ref(case, K):
    import scipy.sparse as sp
    J = sp.csr_matrix(sp.identity(case.n) / case.w.tau + K)       # alpha M + beta K
    return krylov.ilu0_stencil(case.w.dims, J)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ilu0_apply_full_size(P, ctx, slab_case, prec):
    """ILU(0) in natural order on the 128^3 inner operator (the row-of-tiles
    sweep the bench runs), against the oracle's hyperplane elimination."""
    import torch
    case, K, A1, A2 = slab_case
    n, s = case.n, case.s
    X = synth.uniform(33, n * s).reshape(n, s)
    ref = krylov.ilu0_stencil_apply(case.w.dims, _ilu_ref(case, K), X)
    if prec == "fp64":
        Z = torch.empty(n, s, device="cuda", dtype=torch.float64)
        P.pint_precond_apply(ctx, case.op, P.PINT_PC_ILU0, _dev(X), Z)
        np.testing.assert_allclose(Z.cpu().numpy(), ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
    else:
        X32 = X.astype(np.float32)
        Z = torch.empty(n, s, device="cuda", dtype=torch.float32)
        P.pint_ilu0_apply_f32(ctx, case.op, _dev(X32, torch.float32), Z)
        err = np.linalg.norm(Z.cpu().numpy().astype(np.float64) - ref, axis=0)
        # float32 factors and sweeps: a few units of 2^-24 per level of the
        # 382-plane recurrence in an M-matrix, well below 1e-4 relative
        assert np.all(err <= 1e-4 * np.linalg.norm(ref, axis=0)), err / np.linalg.norm(ref, axis=0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gram_and_update_full_size_sampled(P, ctx, prec):
    """Block Gram H = [V_1 .. V_30]^T W and W -= [V] H at N = 128^3, s = 8 and
    the restart length 30 (the last Arnoldi step of a cycle), on sampled
    entries that the oracle computes one by one."""
    import torch
    n, s, nb = 128 ** 3, 8, 30
    dt = torch.float32 if prec == "fp32" else torch.float64
    code = P.PINT_FP32 if prec == "fp32" else P.PINT_FP64
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if prec == "fp32" else (lambda a: a)
    rows = np.sort(synth.splitmix64(41, 64) % np.uint64(n)).astype(np.int64)
    Vd = torch.empty(nb, n, s, device="cuda", dtype=dt)
    cols = []
    Vrows = np.empty((nb, len(rows), s))
    pick = [(b, i) for b in (0, 7, 29) for i in (0, 5)]
    for b in range(nb):
        Vb = cast(synth.uniform(100 + b, n * s).reshape(n, s))
        Vd[b].copy_(torch.from_numpy(Vb))
        Vrows[b] = Vb[rows]
        for bb, i in pick:
            if bb == b:
                cols.append(Vb[:, i].copy())
    W = cast(synth.uniform(99, n * s).reshape(n, s))
    Wd = _dev(W, dt)
    H = torch.empty(nb * s, s, device="cuda", dtype=torch.float64)
    P.pint_block_gram(ctx, code, n, s, nb, Vd, Wd, H)
    Hh = H.cpu().numpy()
    eps = 1e-5 if prec == "fp32" else 1e-13
    for (b, i), v in zip(pick, cols):
        ref = v @ W
        bound = np.abs(v) @ np.abs(W)
        # float32 products are exact in float64; the error is the rounding of
        # float32 partial sums (short chains per thread), relative to sum |v w|
        assert np.all(np.abs(Hh[b * s + i] - ref) <= eps * bound), (b, i)
    Hs = synth.uniform(98, nb * s * s).reshape(nb * s, s) * 0.05
    P.pint_block_update(ctx, code, n, s, nb, Vd, _dev(Hs), Wd)
    got = Wd[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Vm = np.concatenate([Vrows[b] for b in range(nb)], axis=1)
    ref = W[rows] - Vm @ Hs
    bound = np.abs(W[rows]) + np.abs(Vm) @ np.abs(Hs)
    assert np.all(np.abs(got - ref) <= (4e-7 if prec == "fp32" else 1e-15) * nb * s * bound)


@pytest.mark.parametrize("workload", ["diffreact", "richards"])
def test_pipeline_full_size_stage_equations(P, ctx, workload):
    """Algorithm 1 as the bench runs it (512^2 SDIRK2 window s = 2 over 8
    stages; 96^3 implicit Euler window s = 8 over 8 steps): every stored
    stage satisfies its sequential stage equation, recomputed by the oracle
    from the stored stages, to the outer tolerance relative to ||B0||."""
    case = bench.PipelineCase(P, ctx, bench.parse(["--workload", workload]))
    try:
        st = case.step()
        assert st.status == P.PINT_OK
        out = case.out.cpu().numpy()
        n = case.n
        if workload == "diffreact":
            prob = newton.DiffReactProblem((int(round(np.sqrt(n))),) * 2 + (1,))
        else:
            m = int(round(n ** (1 / 3)))
            dims = (m, m, m)
            w = synth.richards_3d(m, case.s)
            Ks = np.exp(2.0 * synth.correlated_field(w.seed_coef, dims[::-1], 8.0 * m / 96.0))
            prob = newton.RichardsProblem(dims, Ks, fv.VanGenuchten(1.0, 2.0, 0.05, 0.4),
                                          1.0 / 16.0)
        stages, fvals = {}, {}
        worst = 0.0
        for g in range(case.G):
            A1, A2, terms, times = coupling.window_matrices(case.A, case.c, case.tau, g, 1)
            B0 = newton.window_B0(prob, terms, stages, fvals, case.y0, 1)
            R = newton.window_residual(prob, A1, A2, times, out[:, g:g + 1], B0)
            rel = np.linalg.norm(R) / np.linalg.norm(B0)
            worst = max(worst, rel)
            stages[g] = out[:, g].copy()
            fvals[g] = prob.f(times[0], out[:, g])
        assert worst <= case.tol * 1.01, worst
    finally:
        case.close()


@pytest.fixture(scope="module")
def seq48():
    """The 48^3 convection-diffusion workload (bench's recipe: log-normal D,
    v = (1, 0.5, 0), tau = 1e-3) stepped sequentially by the oracle over 16
    implicit-Euler steps, each stage equation solved to a relative residual
    of 1e-15."""
    w = synth.convdiff_3d(48, 16)
    D = synth.diffusion_field(w)
    K = fv.convdiff_matrix(w.dims, D, w.velocity)
    B = synth.rhs_block(w)
    A, _, _ = coupling.implicit_euler()
    Y = slab.sequential_dirk_linear(K, np.ones(w.n), A, w.tau, np.zeros(w.n), B, rtol=1e-15)
    return B, Y


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s", [8, 16])
def test_slab_elementwise_equals_sequential_48cube(P, ctx, seq48, s, prec):
    """bench's slab configuration (ILU(0) row-of-tiles sweeps, block
    GMRES(30), default inner tolerances, narrowed inner solves; the Gram
    products on 2 x 152 CTAs) at 48^3 with s = 8 and s = 16, solved to
    tol 1e-13: every column equals sequential stepping (the first s steps of
    the same right-hand sides) to 1e-10 relative in FP64 and 1e-8 with FP32
    inner solves under FP64 refinement."""
    import torch
    B16, Yseq = seq48
    case = bench.LinearCase(P, ctx, bench.parse(["--n", "48", "--s", str(s),
                                                 "--precision", prec]))
    try:
        case.o.tol = 1e-13
        case.Bd.copy_(torch.tensor(np.ascontiguousarray(B16[:, :s]), device="cuda"))
        st = case.step()
        assert st.status == P.PINT_OK
        Yg = case.Y.cpu().numpy()
        ref = Yseq[:, :s]
        err = np.linalg.norm(Yg - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.all(err <= (1e-10 if prec == "fp64" else 1e-8)), err
    finally:
        case.close()
