"""The tensor-core GEMM (tcgen05.mma, BF16 in, FP32 accumulate) against a
plain PyTorch FP32 matmul of the same BF16 inputs."""
import pytest

torch = pytest.importorskip("torch")

import paper_2501_03322_gb300 as P  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (4096, 256, 256), (256, 256, 4096)])
def test_gemm_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = P.gemm_bf16(A, B)
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    # FP32 accumulation of K products of bf16 values: only summation order differs
    err = (C - ref).abs().max().item()
    assert err <= 1e-5 * K ** 0.5 * ref.abs().max().item() + 1e-4, err


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(P.TwError):
        P.gemm_bf16(A, A)
