"""pint_block_gram_noalloc: the Gram product for callers that cannot allocate
device memory (it uses a fixed device array instead of a context's buffers).

Each case runs two calls in a row with different inputs, so that contents left
in the shared array by the first call cannot leak into the second, and checks
H against the definition V^T W evaluated by numpy in float64 (from the same
rounded inputs) and against pint_block_gram. Tolerance per entry: a multiple
of the unit roundoff times sum_r |V_r||W_r|, the scale of a dot product's
rounding error (1e-13 for float64, 1e-5 for float32 with float32 products and
per-thread float32 sums). This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-13, "fp32": 1e-5}


def _noalloc(P, code, n, s, nb, V, W, H):
    import torch
    return P.lib.pint_block_gram_noalloc(code, n, s, nb, ctypes.c_void_p(V.data_ptr()),
                                         ctypes.c_void_p(W.data_ptr()),
                                         ctypes.c_void_p(H.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec,s,nb,n", [("fp64", 8, 7, 5003), ("fp32", 16, 16, 5003),
                                         ("fp64", 3, 5, 5003), ("fp32", 8, 9, 4096),
                                         ("fp64", 2, 300, 4096)])
def test_gram_noalloc_matches_definition_twice(prec, s, nb, n):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_02117_gb300 as P
    dt = torch.float64 if prec == "fp64" else torch.float32
    code = P.PINT_FP64 if prec == "fp64" else P.PINT_FP32
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
            rc = _noalloc(P, code, n, s, nb, V, W, H)
            assert rc == P.PINT_OK, P.pint_last_error(None)
            torch.cuda.synchronize()
            Vh = V.cpu().double().numpy().transpose(0, 2, 1).reshape(nb * s, n)
            Wh = W.cpu().double().numpy()
            exact = Vh @ Wh
            scale = np.abs(Vh) @ np.abs(Wh)
            Hg = H.cpu().numpy()
            assert np.all(np.abs(Hg - exact) <= REL[prec] * scale), \
                f"call {call}: max err {np.max(np.abs(Hg - exact) / scale):.2e} of the scale"
            assert np.all(np.abs(Hg - Href.cpu().numpy()) <= 2 * REL[prec] * scale)
    finally:
        P.pint_destroy(ctx)


def test_gram_noalloc_rejects_sizes_beyond_the_limits():
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
    # nb*s = 1025 basis columns: within the scratch (1025 <= 4096) but wider
    # than one Gram CTA covers
    V = torch.zeros(1025 * 16, device="cuda", dtype=torch.float64)
    W = torch.zeros(16, device="cuda", dtype=torch.float64)
    H = torch.zeros(1025, device="cuda", dtype=torch.float64)
    with pytest.raises(P.PintError) as ei:
        P.pint_block_gram_noalloc(P.PINT_FP64, 16, 1, 1025, V, W, H)
    assert ei.value.code == P.PINT_ERR_INVALID
    assert "1024" in P.pint_last_error(None)
