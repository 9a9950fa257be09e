"""The tensor-core BF16 GEMM (tcgen05, float32 accumulation) against a float64
matrix product of the same bf16 operands on the CPU: tiles with ragged M, N not a
multiple of the tile, bias, ReLU, bf16 and float32 outputs, split-K."""
import numpy as np
import pytest

from tests.gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    require_gpu()
    from paper_2107_05509_gb300 import binding as B
    return B, B.Context(8, 8, 8, 1, 8, 8)


CASES = [
    # M, N, K, splits, relu, bf16 out
    (128, 64, 64, 1, False, False),
    (1, 16, 64, 1, False, False),
    (300, 61, 128, 1, True, False),
    (1000, 128, 640, 1, True, True),
    (257, 32, 192, 1, False, True),
    (130, 80, 1152, 3, True, False),
    (77, 200, 256, 2, False, True),
    (4096, 128, 576, 1, True, True),
]


@pytest.mark.parametrize("M,N,K,splits,relu,bf16", CASES)
def test_gemm_matches_float64(env, M, N, K, splits, relu, bf16):
    B, ctx = env
    g = torch.Generator().manual_seed(M * 7 + N * 13 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    ref = A.double().numpy() @ Bm.double().numpy().T + bias.double().numpy()
    if relu:
        ref = np.maximum(ref, 0.0)
    C = torch.full((M, N), 7.0, dtype=torch.bfloat16 if bf16 else torch.float32, device="cuda")
    buf = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
    B.hr_gemm_bf16(ctx, A.cuda(), Bm.cuda(), C, bias.cuda(), relu, splits, buf)
    got = C.float().cpu().numpy().astype(np.float64)
    # float32 accumulation of K products of size ~1: |error| ~ sqrt(K) * 2^-24 * |terms|
    tol = 1e-5 * np.sqrt(K) * np.sqrt(K) + 1e-6
    if bf16:
        tol = np.maximum(tol, 2.0 ** -8 * np.abs(ref))   # one bf16 rounding of the result
    err = np.abs(got - ref)
    assert (err <= tol).all(), (np.argwhere(err > tol)[:5], err.max())
    assert B.hr_get_status(ctx) == B.HR_OK
