"""GPU parity of the batched persistent slab solver (pint_solve_batch): many
slab solves of uneven N and s in one launch, each solved inside one cluster
of CTAs by global GMRES on the unsplit operator of Eq.
general-system-time-steps. Every queued solve must equal sequential
one-step-at-a-time implicit Euler (FP64 bar 1e-10 per column at tol 1e-13),
meet the stopping test in the oracle's own float64 residual, agree with its
solo pint_solve_block (PINT_SOLVER_GLOBAL) solve, and give bitwise the same
result alone and in the mix."""
import numpy as np
import pytest

import synth
from oracle import coupling, fv, slab

pytestmark = pytest.mark.gpu

# (dims, s): uneven sizes and block widths, one of them smaller than a warp
JOBS = [((24, 24, 1), 4), ((10, 9, 8), 2), ((40, 33, 1), 8), ((12, 12, 12), 16),
        ((7, 5, 1), 1), ((30, 20, 1), 3)]
TAU = 1e-3
V = (1.0, 0.5, 0.0)


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _colerr(Y, Yref):
    return np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)


def _make(P, ctx, specs, seed0=50):
    """One operator per job (its own diffusion field and coupling)."""
    jobs = []
    for q, (dims, s) in enumerate(specs):
        n = int(np.prod(dims))
        D = np.exp(synth.normal(seed0 + q, n)).reshape(dims[::-1])
        K = fv.convdiff_matrix(dims, D, V)
        op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), V)
        A, _, _ = coupling.implicit_euler()
        A1, A2, _ = coupling.multistep_matrices(A, s, TAU)
        P.pint_set_coupling(ctx, op, A1, A2)
        B = synth.uniform(seed0 + 100 + q, n * s).reshape(n, s)
        jobs.append(dict(op=op, K=K, n=n, s=s, A=A, A1=A1, A2=A2, B=B))
    return jobs


def _free(P, jobs):
    for j in jobs:
        P.pint_operator_destroy(j["op"])


def _opts(P, tol, pc="jacobi"):
    o = P.pint_opts_default()
    o.tol = tol
    o.precision = P.PINT_FP64
    o.precond = {"none": P.PINT_PC_NONE, "jacobi": P.PINT_PC_JACOBI}[pc]
    return o


def _run(P, ctx, jobs, o, cluster, idx=None, threads=0):
    import torch
    idx = range(len(jobs)) if idx is None else idx
    Ys = {i: torch.zeros(jobs[i]["n"], jobs[i]["s"], device="cuda", dtype=torch.float64)
          for i in idx}
    Bs = {i: _dev(jobs[i]["B"]) for i in idx}
    sts = P.pint_solve_batch(ctx, [(jobs[i]["op"], Bs[i], None, Ys[i]) for i in idx], o,
                             cluster_ctas=cluster, cta_threads=threads)
    return {i: Ys[i].cpu().numpy() for i in idx}, dict(zip(idx, sts))


@pytest.mark.parametrize("cluster,threads", [(1, 512), (1, 256), (1, 128), (2, 512),
                                             (4, 256), (16, 512)])
def test_batch_equals_sequential_stepping(P, ctx, cluster, threads):
    """Every job of one launch equals sequential implicit Euler to 1e-10 per
    column (both at relative residual 1e-13), for several cluster sizes and
    CTA widths."""
    jobs = _make(P, ctx, JOBS)
    try:
        Y, st = _run(P, ctx, jobs, _opts(P, 1e-13), cluster, threads=threads)
        for i, j in enumerate(jobs):
            assert st[i].status == P.PINT_OK, (i, st[i].as_dict(j["s"]))
            assert st[i].kernel_launches == 1
            Yref = slab.sequential_dirk_linear(j["K"], np.ones(j["n"]), j["A"], TAU,
                                               np.zeros(j["n"]), j["B"])
            err = _colerr(Y[i], Yref)
            assert np.all(err < 1e-10), (i, err)
    finally:
        _free(P, jobs)


def _ortho(cluster):
    """One CTA per job orthogonalises by modified Gram-Schmidt, a cluster by
    two classical passes."""
    return "mgs" if cluster == 1 else "cgs2"


@pytest.mark.parametrize("cluster", [1, 4])
def test_batch_meets_tol_in_oracle_residual_and_matches_solo(P, ctx, cluster):
    """At tol 1e-10 each job meets ||R_k|| <= tol ||F_k|| in the oracle's
    float64 residual, its reported relative residuals match the oracle's, and
    it agrees with the solo PINT_SOLVER_GLOBAL + Jacobi solve of the same job
    to the accuracy both guarantee; the Arnoldi step count is within one step
    per restart of the oracle's global GMRES with the same orthogonalisation."""
    import torch
    tol = 1e-10
    jobs = _make(P, ctx, JOBS, seed0=80)
    try:
        Y, st = _run(P, ctx, jobs, _opts(P, tol), cluster)
        for i, j in enumerate(jobs):
            n, s = j["n"], j["s"]
            R = slab.coupled_residual(j["K"], np.ones(n), j["A1"], j["A2"], Y[i], B=j["B"])
            F = slab.rhs_F(j["A2"], B=j["B"])
            rel = np.linalg.norm(R, axis=0) / np.linalg.norm(F, axis=0)
            assert np.all(rel <= tol * (1 + 1e-6)), (i, rel)
            np.testing.assert_allclose(st[i].as_dict(s)["col_relres"], rel, rtol=1e-4,
                                       atol=1e-16)
            o = _opts(P, tol)
            o.solver = P.PINT_SOLVER_GLOBAL
            Ys = torch.zeros(n, s, device="cuda", dtype=torch.float64)
            P.pint_solve_block(ctx, j["op"], _dev(j["B"]), None, Ys, o,
                               raise_on_nonconvergence=True)
            Yd = slab.solve_all_at_once_dense(j["K"], np.ones(n), j["A1"], j["A2"], j["B"]) \
                if n * s <= 3000 else None
            if Yd is not None:
                assert np.all(_colerr(Y[i], Yd) < 1e-7), i
            assert np.all(_colerr(Y[i], Ys.cpu().numpy()) < 1e-7), i
            _, info = slab.slab_solve_global(j["K"], np.ones(n), j["A1"], j["A2"], j["B"],
                                             tol=tol, precond="jacobi", restart=30,
                                             ortho=_ortho(cluster))
            assert abs(st[i].inner_its - info["inner"]) <= 1 + info["cycles"], \
                (i, st[i].inner_its, info)
    finally:
        _free(P, jobs)


@pytest.mark.parametrize("cluster,threads", [(1, 256), (4, 512)])
def test_batch_alone_equals_in_mix_bitwise(P, ctx, cluster, threads):
    """A job's result and iteration counts do not depend on the other jobs of
    the launch: each job alone gives bitwise the Y it gets in the mix (same
    cluster size and CTA width)."""
    jobs = _make(P, ctx, JOBS, seed0=110)
    try:
        o = _opts(P, 1e-10)
        Ymix, smix = _run(P, ctx, jobs, o, cluster, threads=threads)
        for i in range(len(jobs)):
            Y1, s1 = _run(P, ctx, jobs, o, cluster, idx=[i], threads=threads)
            assert np.array_equal(Y1[i], Ymix[i]), i
            assert (s1[i].inner_its, s1[i].outer_its) == (smix[i].inner_its, smix[i].outer_its)
    finally:
        _free(P, jobs)


def test_batch_shared_operator_b0_and_no_preconditioner(P, ctx):
    """Two jobs on one operator with different right-hand sides, a B0 term
    (theta method with its explicit first stage eliminated), and
    preconditioner none: each equals the dense all-at-once solve."""
    import torch
    dims, s = (6, 5, 4), 3
    n = int(np.prod(dims))
    D = np.exp(synth.normal(140, n)).reshape(dims[::-1])
    K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.25))
    A, _, _ = coupling.theta_method(0.5)
    A1, A2, _ = coupling.multistep_matrices(A, s, 1e-2, eliminate_first=True)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, 0.5, 0.25))
    try:
        P.pint_set_coupling(ctx, op, A1, A2)
        Bs = [synth.uniform(141 + q, n * s).reshape(n, s) for q in range(2)]
        B0s = [synth.uniform(151 + q, n * s).reshape(n, s) for q in range(2)]
        for pc in ("none", "jacobi"):
            Ys = [torch.zeros(n, s, device="cuda", dtype=torch.float64) for _ in range(2)]
            dB = [_dev(b) for b in Bs]
            dB0 = [_dev(b) for b in B0s]
            st = P.pint_solve_batch(ctx, [(op, dB[q], dB0[q], Ys[q]) for q in range(2)],
                                    _opts(P, 1e-13, pc), cluster_ctas=2,
                                    raise_on_nonconvergence=True)
            for q in range(2):
                Yd = slab.solve_all_at_once_dense(K, np.ones(n), A1, A2, Bs[q], B0s[q])
                assert np.all(_colerr(Ys[q].cpu().numpy(), Yd) < 1e-10), (pc, q)
                assert st[q].status == P.PINT_OK
    finally:
        P.pint_operator_destroy(op)


def test_batch_zero_rhs_nonconvergence_and_invalid_arguments(P, ctx):
    import torch
    jobs = _make(P, ctx, JOBS[:2], seed0=160)
    try:
        j0, j1 = jobs
        # F = 0 and Y = 0: converged before any Arnoldi step (absolute tol)
        Y0 = torch.zeros(j0["n"], j0["s"], device="cuda", dtype=torch.float64)
        Y1 = torch.zeros(j1["n"], j1["s"], device="cuda", dtype=torch.float64)
        o = _opts(P, 1e-14)
        o.max_outer = 1
        o.restart = 2
        st = P.pint_solve_batch(ctx, [(j0["op"], None, None, Y0),
                                      (j1["op"], _dev(j1["B"]), None, Y1)], o)
        assert st[0].status == P.PINT_OK and st[0].outer_its == 0 and st[0].inner_its == 0
        assert float(Y0.abs().max()) == 0.0
        # one restart of GMRES(2) cannot reach 1e-14: reported, not raised
        assert st[1].status == P.PINT_ERR_NOT_CONVERGED
        assert st[1].outer_its == 1 and st[1].inner_its == 2
        assert max(st[1].as_dict(j1["s"])["col_relres"]) > 1e-14
        assert bool(torch.isfinite(Y1).all())
        with pytest.raises(P.PintError) as ei:
            P.pint_solve_batch(ctx, [(j1["op"], _dev(j1["B"]), None, Y1)], o,
                               raise_on_nonconvergence=True)
        assert ei.value.code == P.PINT_ERR_NOT_CONVERGED
        bad = []
        o2 = _opts(P, 1e-10)
        o2.precision = P.PINT_FP32
        bad.append((o2, 0, 0))
        o3 = _opts(P, 1e-10)
        o3.precond = P.PINT_PC_ILU0
        bad.append((o3, 0, 0))
        bad.append((_opts(P, 1e-10), 17, 0))
        bad.append((_opts(P, 1e-10), -1, 0))
        bad.append((_opts(P, 1e-10), 1, 384))
        o4 = _opts(P, 1e-10)
        o4.restart = 40                        # at most 32 in the batched solver
        bad.append((o4, 1, 0))
        for ob, c, t in bad:
            with pytest.raises(P.PintError) as ei:
                P.pint_solve_batch(ctx, [(j0["op"], None, None, Y0)], ob, cluster_ctas=c,
                                   cta_threads=t)
            assert ei.value.code == P.PINT_ERR_INVALID
        assert P.pint_batch_auto_cluster(ctx, [(j1["op"], None, None, Y1)]) == 2   # 720 rows
        assert P.pint_batch_auto_cluster(ctx, [(j0["op"], None, None, Y0)] * 500) == 1
        assert P.pint_batch_auto_threads(ctx, 10000, 1) == 512
        assert P.pint_batch_auto_threads(ctx, 1, 16) == 256
    finally:
        _free(P, jobs)


def test_batch_c1_size_against_oracle(P, ctx):
    """The 64 x 64 convection-diffusion slab (s = 4, Jacobi, tol 1e-10) with
    the automatic cluster size, alone and as 32 copies with different
    right-hand sides: each meets tol in the oracle residual and equals the
    oracle's global GMRES solution (same orthogonalisation) to 1e-7 relative
    per column."""
    import torch
    dims, s = (64, 64, 1), 4
    n = 64 * 64
    D = np.ones((1, 64, 64))
    K = fv.convdiff_matrix(dims, D, V)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), V)
    try:
        A, _, _ = coupling.implicit_euler()
        A1, A2, _ = coupling.multistep_matrices(A, s, TAU)
        P.pint_set_coupling(ctx, op, A1, A2)
        for copies in (1, 32):
            Bs = [synth.uniform(170 + q, n * s).reshape(n, s) for q in range(copies)]
            Ys = [torch.zeros(n, s, device="cuda", dtype=torch.float64) for _ in Bs]
            dB = [_dev(b) for b in Bs]
            st = P.pint_solve_batch(ctx, [(op, dB[q], None, Ys[q]) for q in range(copies)],
                                    _opts(P, 1e-10), raise_on_nonconvergence=True)
            cl = P.pint_batch_auto_cluster(ctx, [(op, dB[q], None, Ys[q])
                                                 for q in range(copies)])
            assert cl == (16 if copies == 1 else 8)
            for q in (0, copies - 1):
                Y = Ys[q].cpu().numpy()
                R = slab.coupled_residual(K, np.ones(n), A1, A2, Y, B=Bs[q])
                F = slab.rhs_F(A2, B=Bs[q])
                assert np.all(np.linalg.norm(R, axis=0) <= 1e-10 * (1 + 1e-6) *
                              np.linalg.norm(F, axis=0))
                Yo, info = slab.slab_solve_global(K, np.ones(n), A1, A2, Bs[q], tol=1e-10,
                                                  precond="jacobi", restart=30,
                                                  ortho=_ortho(cl))
                assert np.all(_colerr(Y, Yo) < 1e-7)
                assert abs(st[q].inner_its - info["inner"]) <= 1 + info["cycles"]
    finally:
        P.pint_operator_destroy(op)


@pytest.mark.parametrize("cluster,threads", [(1, 512), (16, 256)])
def test_batch_plan_replays_the_captured_graph(P, ctx, cluster, threads):
    """The resident plan (descriptors, workspace and a captured CUDA graph made
    once): a replay gives bitwise the result of the first run and of the
    one-shot pint_solve_batch with the same shape; new right-hand sides written
    into the same buffers are solved on the next replay (each equals
    sequential stepping); the plan reports the launch shape it took."""
    import torch
    jobs = _make(P, ctx, JOBS[:4], seed0=190)
    try:
        o = _opts(P, 1e-13)
        Ys = [torch.zeros(j["n"], j["s"], device="cuda", dtype=torch.float64) for j in jobs]
        Bs = [_dev(j["B"]) for j in jobs]
        plan = P.BatchPlan(ctx, [(j["op"], Bs[q], None, Ys[q]) for q, j in enumerate(jobs)], o,
                           cluster_ctas=cluster, cta_threads=threads)
        try:
            sh = plan.shape()
            assert (sh["cluster_ctas"], sh["cta_threads"]) == (cluster, threads)
            assert 1 <= sh["resident_clusters"] <= len(jobs)
            st1 = plan.run(raise_on_nonconvergence=True)
            Y1 = [y.cpu().numpy() for y in Ys]
            for y in Ys:
                y.zero_()
            st2 = plan.run(raise_on_nonconvergence=True)
            for q in range(len(jobs)):
                assert np.array_equal(Ys[q].cpu().numpy(), Y1[q])
                assert st1[q].inner_its == st2[q].inner_its
            Yo, _ = _run(P, ctx, jobs, o, cluster, threads=threads)
            for q in range(len(jobs)):
                assert np.array_equal(Yo[q], Y1[q])
            # new right-hand sides in the same device buffers
            newB = [synth.uniform(200 + q, j["n"] * j["s"]).reshape(j["n"], j["s"])
                    for q, j in enumerate(jobs)]
            for q in range(len(jobs)):
                Bs[q].copy_(torch.as_tensor(newB[q]))
                Ys[q].zero_()
            plan.run(raise_on_nonconvergence=True)
            for q, j in enumerate(jobs):
                Yref = slab.sequential_dirk_linear(j["K"], np.ones(j["n"]), j["A"], TAU,
                                                   np.zeros(j["n"]), newB[q])
                assert np.all(_colerr(Ys[q].cpu().numpy(), Yref) < 1e-10), q
        finally:
            plan.close()
        with pytest.raises(P.PintError) as ei:
            o2 = _opts(P, 1e-10)
            o2.precond = P.PINT_PC_ILU0
            P.BatchPlan(ctx, [(jobs[0]["op"], Bs[0], None, Ys[0])], o2)
        assert ei.value.code == P.PINT_ERR_INVALID
    finally:
        _free(P, jobs)


@pytest.mark.parametrize("cluster", [1, 4])
def test_batch_operation_count_follows_its_definition(P, ctx, cluster):
    """pint_stats.flops of a job equals the algorithmic float64 count of the
    batched method written out (FMA = 2): one GMRES(m) cycle that cannot
    converge (tol 1e-300, max_outer 1) takes exactly m steps; the count adds
    the per-job set-up, three residuals with their column norms, the cycle's
    start, m Arnoldi steps (modified Gram-Schmidt with one CTA per job: 4(j+1)
    N s per step; two classical passes on a cluster: 8(j+1) N s) and the
    correction."""
    import torch
    jobs = _make(P, ctx, [((20, 18, 1), 4)], seed0=230)
    try:
        j = jobs[0]
        n, s, m = j["n"], j["s"], 6
        o = _opts(P, 1e-300)
        o.max_outer = 1
        o.restart = m
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        st = P.pint_solve_batch(ctx, [(j["op"], _dev(j["B"]), None, Y)], o,
                                cluster_ctas=cluster)[0]
        assert (st.outer_its, st.inner_its, st.restarts) == (1, m, 1)
        nnz = int(P.pint_operator_nnz(j["op"]))
        nA = int(np.count_nonzero(j["A1"]) + np.count_nonzero(j["A2"]))
        ns = n * s
        c_pre = 2 * nnz * s + 2 * n * nA + 2 * ns
        c_res = c_pre + ns                                # B given, no B0
        k = 4 if cluster == 1 else 8
        steps = sum(c_pre + k * (i + 1) * ns + 3 * ns for i in range(m))
        want = (nnz + n) + 3 * (c_res + 2 * ns) + ns + steps + 2 * m * ns + 2 * ns
        assert st.flops == want
    finally:
        _free(P, jobs)
