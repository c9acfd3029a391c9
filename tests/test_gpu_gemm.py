"""The tensor-core GEMM (tcgen05, BF16 x BF16 -> FP32) against a float64
product of the same BF16 values: products of two BF16 numbers are exact in
FP32, so the only error is FP32 accumulation, bounded by K * 2^-24 times the
sum of |a_ik b_jk|."""

import numpy as np
import pytest
import torch

from paper_1610_07159_gb300 import sf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sf.load()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("M,N,K,BN,splits", [
    (128, 16, 64, 16, 1),     # one tile, one chunk
    (200, 64, 576, 64, 1),    # ragged M, nine chunks
    (1000, 256, 320, 128, 1), # two N tiles
    (77, 32, 1024, 32, 4),    # split K
    (300, 48, 128, 48, 3),    # N not a power of two; one split without work
])
def test_gemm_matches_float64_product(M, N, K, BN, splits):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = sf.gemm_bf16(A.cuda(), B.cuda(), BN=BN, splits=splits).cpu().double().numpy()
    a, b = A.double().numpy(), B.double().numpy()
    kc = -(-(K // 64) // splits)
    ref = np.zeros((splits, M, N))
    bound = np.zeros((splits, M, N))
    for s in range(splits):
        k0, k1 = min(K, s * kc * 64), min(K, (s + 1) * kc * 64)
        ref[s] = a[:, k0:k1] @ b[:, k0:k1].T
        bound[s] = np.abs(a[:, k0:k1]) @ np.abs(b[:, k0:k1]).T
    err = np.abs(C - ref)
    assert np.all(err <= K * 2.0 ** -24 * bound + 1e-30), float(np.max(err / (bound + 1e-30)))


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(10, 60, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 60, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sf.SFError):
        sf.gemm_bf16(A, B)  # K not a multiple of 64
    A = torch.zeros(10, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(20, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(sf.SFError):
        sf.gemm_bf16(A, B)  # N not a multiple of 16
