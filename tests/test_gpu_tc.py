"""The tensor-core contraction (kfbi_tc_gemm: tcgen05 MMAs, accumulator in tensor memory)
against a float64 matrix product of the same float32 inputs.

With every input split into two bfloat16 terms and three products accumulated in float32, each
product carries about 2^-16 relative error; over K terms of random sign the sum's error stays
within 1e-4 of the largest |C|. With B exact in bfloat16 and A in three terms (terms = 4) only
float32 accumulation remains: 1e-5. The plain bfloat16 product (terms = 1) is held to 1e-2.
Shapes cover full tiles, ragged edges in M, N and K, both operand orders, and N below 32.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_01068_gb300.kfbi")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_01068_gb300 import build

    build.build()
    K.load()


@pytest.mark.parametrize("M,N,Kd,ta,tb", [(128, 256, 256, False, False), (128, 128, 128, False, True),
                                          (200, 100, 77, True, False), (64, 24, 16, True, True),
                                          (513, 256, 300, False, False)])
@pytest.mark.parametrize("terms,tol", [(3, 1e-4), (1, 1e-2), (4, 1e-5), (6, 1e-5)])
def test_tc_gemm_matches_float64_product(M, N, Kd, ta, tb, terms, tol):
    g = torch.Generator(device="cpu").manual_seed(M + N + Kd)
    A = torch.randn((Kd, M) if ta else (M, Kd), generator=g, dtype=torch.float32).cuda()
    B = torch.randn((Kd, N) if tb else (N, Kd), generator=g, dtype=torch.float32).cuda()
    if terms == 4:  # B exact in bfloat16, A in three terms
        B = B.to(torch.bfloat16).to(torch.float32)
    C, err = K.tc_gemm(A, B, transA=ta, transB=tb, terms=terms)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ad = (A.t() if ta else A).double()
    Bd = (B.t() if tb else B).double()
    ref = Ad @ Bd.t()
    e = float((C.double() - ref).abs().max() / ref.abs().max())
    print(f"tc_gemm {M}x{N}x{Kd} ta={ta} tb={tb} terms={terms}: max error / max |C| = {e:.2e}")
    assert e < tol
