"""pint_block_gram_noalloc: the Gram product for callers that cannot allocate
device memory (it uses a fixed device array instead of a context's buffers).
Checked against pint_block_gram on two calls in a row, with different inputs,
so that contents left in the shared array by the first call cannot leak into
the second. This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,s,nb", [("fp64", 8, 7), ("fp32", 16, 16), ("fp64", 3, 5)])
def test_gram_noalloc_matches_gram_twice(prec, s, nb):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02117_gb300 as P
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
    n = 5003
    ctx = P.pint_create(0)
    try:
        for call in range(2):
            V = torch.tensor(synth.uniform(20 + call, nb * n * s).reshape(nb, n, s), device="cuda",
                             dtype=dt)
            W = torch.tensor(synth.uniform(30 + call, n * s).reshape(n, s), device="cuda",
                             dtype=dt)
            Href = torch.empty(nb * s, s, device="cuda", dtype=torch.float64)
            H = torch.full((nb * s, s), float("nan"), device="cuda", dtype=torch.float64)
            P.pint_block_gram(ctx, code, n, s, nb, V, W, Href)
            rc = P.lib.pint_block_gram_noalloc(code, n, s, nb, ctypes.c_void_p(V.data_ptr()),
                                               ctypes.c_void_p(W.data_ptr()),
                                               ctypes.c_void_p(H.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == P.PINT_OK, P.pint_last_error(None)
            torch.cuda.synchronize()
            tol = 1e-12 if prec == "fp64" else 2e-5
            np.testing.assert_allclose(H.cpu().numpy(), Href.cpu().numpy(), rtol=0,
                                       atol=tol * np.sqrt(n))
    finally:
        P.pint_destroy(ctx)


def test_gram_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02117_gb300 as P
    V = torch.zeros(17 * 16 * 16, device="cuda", dtype=torch.float64)
    W = torch.zeros(16 * 16, device="cuda", dtype=torch.float64)
    H = torch.zeros(17 * 16 * 16, device="cuda", dtype=torch.float64)
    with pytest.raises(P.PintError) as ei:
        P.pint_block_gram_noalloc(P.PINT_FP64, 16, 16, 17, V, W, H)     # 17*16*16 > 4096
    assert ei.value.code == P.PINT_ERR_INVALID
    assert "exceeds the maximum" in P.pint_last_error(None)
