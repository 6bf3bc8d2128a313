"""The BF16 tensor-core GEMM (tcgen05, TMA, tensor memory) behind the neural-field training:
C = A B^T for bf16 operands with FP32 accumulation, against an FP64 product of the same
bf16 values. Only the summation order differs, so the tolerance is a few FP32 ulps of the
accumulated magnitude."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")
torch = pytest.importorskip("torch")


def _ref(A, B):
    return A.double().cpu().numpy() @ B.double().cpu().numpy().T


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 256), (384, 512, 1024), (128, 128, 192),
                                   (1024, 256, 256)])
def test_gemm_matches_fp64_product(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.zeros(M, N, device="cuda")
    gcpush.gemm_bf16_tn(A, B, C)
    torch.cuda.synchronize()
    ref = _ref(A, B)
    scale = np.sqrt(K)
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=0, atol=1e-4 * scale)


def test_gemm_split_k_accumulates():
    M, N, K = 256, 256, 8192
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), 0.5, device="cuda")
    gcpush.gemm_bf16_tn(A, B, C, split_k=16, accumulate=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(C.cpu().numpy(), _ref(A, B) + 0.5, rtol=0, atol=2e-4 * np.sqrt(K))


def test_gemm_rejects_bad_shapes():
    A = torch.zeros(100, 64, device="cuda", dtype=torch.bfloat16)
    B = torch.zeros(128, 64, device="cuda", dtype=torch.bfloat16)
    C = torch.zeros(100, 128, device="cuda")
    with pytest.raises(gcpush.GcError):
        gcpush.gemm_bf16_tn(A, B, C)


@pytest.mark.parametrize("a_mn,b_mn", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(128, 256, 128), (256, 128, 320)])
def test_gemm_mn_major_operands(a_mn, b_mn, M, N, K):
    """Operands stored transposed (MN-major shared-memory layout through TMA)."""
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 5 * K + 11 * a_mn + 13 * b_mn)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.zeros(M, N, device="cuda")
    gcpush.gemm_bf16(A.t().contiguous() if a_mn else A, B.t().contiguous() if b_mn else B, C,
                     a_mn=bool(a_mn), b_mn=bool(b_mn))
    torch.cuda.synchronize()
    np.testing.assert_allclose(C.cpu().numpy(), _ref(A, B), rtol=0, atol=1e-4 * np.sqrt(K))


def test_gemm_mn_major_split_k():
    """dW = dZ^T H shape of the training: both operands MN-major, K = batch, split over CTAs."""
    M, N, K = 256, 256, 4096
    g = torch.Generator(device="cuda").manual_seed(5)
    dZ = torch.randn(K, M, device="cuda", generator=g).to(torch.bfloat16)
    H = torch.randn(K, N, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.zeros(M, N, device="cuda")
    gcpush.gemm_bf16(dZ, H, C, a_mn=True, b_mn=True, split_k=8, accumulate=True)
    torch.cuda.synchronize()
    ref = dZ.double().cpu().numpy().T @ H.double().cpu().numpy()
    np.testing.assert_allclose(C.cpu().numpy(), ref, rtol=0, atol=2e-4 * np.sqrt(K))
