"""The tcgen05 BF16 GEMM building block (ctd_gemm_bf16) against a float64 product of the same
BF16 operands.  BF16 x BF16 products are exact in FP32; only the FP32 accumulation rounds, so
the relative error bound is ~K * 2^-24 of the sum of |products|.  Shapes cover every (N, K) the
node MLPs use for F = 64 and F = 128, K that ends in half a 64-column block (zero-filled by the
TMA), ragged M tails, and multiple persistent tiles per CTA."""
import ctypes

import numpy as np
import pytest

from gpu_common import engine

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64), (128, 128), (256, 128), (384, 128), (128, 256), (128, 384), (192, 64), (32, 128),
          (64, 128), (128, 64), (256, 64), (64, 192), (64, 96), (32, 96), (96, 160)]


@pytest.mark.parametrize("N,K", SHAPES)
def test_gemm_bf16_matches_float64(N, K):
    import torch
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    g = torch.Generator(device="cpu").manual_seed(N * 1000 + K)
    pot = eng.Potential(64, T=1, n_species=1)
    try:
        for M in (1, 127, 128, 1000, 40000):
            A = torch.randn(M, K, generator=g).to(torch.bfloat16)
            B = torch.randn(N, K, generator=g).to(torch.bfloat16)
            Ad, Bd = A.cuda(), B.cuda()
            C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            P = lambda t: ctypes.c_void_p(t.data_ptr())
            _lib.ctd_gemm_bf16(pot.ctx, M, N, K, P(Ad), K, P(Bd), P(C), N)
            ref = A.double() @ B.double().T
            bound = (A.double().abs() @ B.double().abs().T) * (K * 2.0 ** -23) + 1e-30
            err = (C.cpu().double() - ref).abs()
            assert bool((err <= bound).all()), f"M={M}: max err {float(err.max()):.3e}"
    finally:
        pot.close()


def test_gemm_bf16_leading_dimension():
    """A read from a wider row-major buffer (lda > K), as the model does for stacked blocks."""
    import torch
    eng = engine()
    from paper_2506_04055_gb300 import _lib
    g = torch.Generator(device="cpu").manual_seed(7)
    M, N, K, lda = 3000, 128, 128, 384
    Afull = torch.randn(M, lda, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    with eng.Potential(64, T=1, n_species=1) as pot:
        Ad, Bd = Afull.cuda(), B.cuda()
        C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        _lib.ctd_gemm_bf16(pot.ctx, M, N, K, P(Ad[:, 128:]), lda, P(Bd), P(C), N)
        ref = Afull[:, 128:256].double() @ B.double().T
        np.testing.assert_allclose(C.cpu().double().numpy(), ref.numpy(), rtol=1e-4, atol=1e-4)
