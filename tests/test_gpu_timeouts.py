"""The bounded device waits give up and report PINT_ERR_TIMEOUT instead of
hanging, and the context stays usable afterwards. Each wait is made to run
out on something nothing completes (a flag nothing stores, an mbarrier
transaction count no copy delivers) with a 1 ms deadline; no kernel traps and
no copy is in flight when it returns."""
import numpy as np
import pytest

import synth
from oracle import coupling, fv, slab

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(P, ctx, which):
    import torch
    assert P.pint_test_wait_timeout(ctx, which, 1.0) == P.PINT_ERR_TIMEOUT
    assert "exceeded its time budget" in P.pint_last_error(ctx)
    # a normal slab solve on the same context (ILU(0): the dependency waits
    # and, n a multiple of 64, the Gram bulk-copy ring both run) is correct
    dims = (16, 16, 16)
    n, s, tau = 16 ** 3, 4, 1e-3
    D = np.exp(synth.normal(41, n)).reshape(16, 16, 16)
    B = synth.uniform(42, n * s).reshape(n, s)
    A, _, _ = coupling.implicit_euler()
    A1, A2, _ = coupling.multistep_matrices(A, s, tau)
    op = P.pint_fv_convdiff(ctx, *dims, D.ravel(), (1.0, 0.5, 0.0))
    try:
        P.pint_set_coupling(ctx, op, A1, A2)
        o = P.pint_opts_default()
        o.tol = 1e-13
        o.precond = P.PINT_PC_ILU0
        Y = torch.zeros(n, s, device="cuda", dtype=torch.float64)
        st = P.pint_solve_block(ctx, op, torch.tensor(B, device="cuda"), None, Y, o)
        assert st.status == P.PINT_OK
        K = fv.convdiff_matrix(dims, D, (1.0, 0.5, 0.0))
        Yref = slab.sequential_dirk_linear(K, np.ones(n), A, tau, np.zeros(n), B)
        err = np.linalg.norm(Y.cpu().numpy() - Yref, axis=0) / np.linalg.norm(Yref, axis=0)
        assert np.all(err < 1e-10), err
    finally:
        P.pint_operator_destroy(op)


def test_bounded_wait_rejects_bad_arguments(P, ctx):
    assert P.pint_test_wait_timeout(ctx, 2, 1.0) == P.PINT_ERR_INVALID
    assert P.pint_test_wait_timeout(ctx, 0, 0.0) == P.PINT_ERR_INVALID
    assert P.pint_test_wait_timeout(ctx, 0, 5000.0) == P.PINT_ERR_INVALID
