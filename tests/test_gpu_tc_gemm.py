"""The tcgen05 contraction engine against torch matmul of the same BF16
inputs (FP32 reference), in both operand modes, with ragged tiles."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_11623_gb300 import _lib
    _lib.load()
    return _lib


def _run(L, A, B, rows, N, K, trans):
    C = torch.full((rows, N), float("nan"), device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    L.fbsde_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), rows, N, K, A.shape[1], B.shape[1], N, trans, st)
    return C


@pytest.mark.parametrize("rows,N,K", [(128, 256, 256), (300, 256, 256), (257, 112, 100), (1, 16, 8),
                                      (1000, 64, 64), (129, 48, 200), (384, 256, 1024)])
def test_nt_mode(L, rows, N, K):
    g = torch.Generator(device="cuda").manual_seed(rows * 7 + N)
    ldk = (K + 7) // 8 * 8
    A = torch.randn(rows, ldk, device="cuda", generator=g).bfloat16()
    B = torch.randn(N, ldk, device="cuda", generator=g).bfloat16()
    C = _run(L, A, B, rows, N, K, 0)
    ref = A[:, :K].float() @ B[:, :K].float().T
    err = (C - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


@pytest.mark.parametrize("rows,N,K", [(256, 256, 1000), (128, 256, 64), (48, 48, 77), (256, 112, 500),
                                      (200, 64, 4096), (16, 16, 1)])
def test_tn_mode(L, rows, N, K):
    g = torch.Generator(device="cuda").manual_seed(rows * 11 + N + K)
    lda = (rows + 7) // 8 * 8
    ldb = (N + 7) // 8 * 8
    A = torch.randn(K, lda, device="cuda", generator=g).bfloat16()
    B = torch.randn(K, ldb, device="cuda", generator=g).bfloat16()
    C = _run(L, A, B, rows, N, K, 1)
    ref = A[:, :rows].float().T @ B[:, :N].float()
    err = (C - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def test_rejects_bad_shapes(L):
    A = torch.zeros(128, 64, device="cuda").bfloat16()
    st = torch.cuda.current_stream().cuda_stream
    C = torch.zeros(128, 24, device="cuda")
    for (N, lda) in [(24, 64), (272, 64), (16, 60)]:
        with pytest.raises(L.FBSDEError) as ei:
            L.fbsde_gemm_bf16(A.data_ptr(), A.data_ptr(), C.data_ptr(), 128, N, 32, lda, 64, 272, 0, st)
        assert ei.value.status == L.FBSDE_ERR_INVALID
