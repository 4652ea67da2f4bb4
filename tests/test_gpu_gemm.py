"""tcgen05 BF16 GEMM (TMEM accumulation) against an FP64 CPU product of the same
BF16-rounded operands: layouts, transposed views, ragged edges, split-K, epilogue."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_15183_gb300 import build, geotrace
    build.build()
    return geotrace.load_library()


def gemm(lib, A, B, M, N, K, a_strides, b_strides, bias=None, act=0, splits=1, bn=128,
         accumulate=False, C=None):
    if C is None:
        C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    rc = lib.gt_gemm_bf16(0, None, M, N, K, ctypes.c_void_p(A.data_ptr()), a_strides[0],
                          a_strides[1], ctypes.c_void_p(B.data_ptr()), b_strides[0], b_strides[1],
                          None if bias is None else ctypes.c_void_p(bias.data_ptr()), act,
                          ctypes.c_void_p(C.data_ptr()), N, int(accumulate), splits, bn)
    assert rc == 0
    torch.cuda.synchronize()
    return C


def ref(A, B, bias=None, act=0):
    a = A.float().cpu().numpy().astype(np.float64)
    b = B.float().cpu().numpy().astype(np.float64)
    z = a @ b.T
    if bias is not None:
        z = z + bias.cpu().numpy().astype(np.float64)
    if act == 1:
        z = z / (1 + np.exp(-z))
    return z


@pytest.mark.parametrize("M,N,K,bn", [(128, 128, 64, 128), (128, 256, 256, 256),
                                      (300, 70, 200, 64), (5, 3, 16, 16), (257, 40, 33, 32)])
def test_gemm_matches_cpu(lib, M, N, K, bn):
    g = torch.Generator().manual_seed(M * 7 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    for act in (0, 1):
        C = gemm(lib, A, B, M, N, K, (K, 1), (K, 1), bias, act, bn=bn)
        R = ref(A, B, bias, act)
        np.testing.assert_allclose(C.cpu().numpy(), R, rtol=1e-4, atol=1e-4 * np.sqrt(K))


def test_gemm_transposed_views_and_split_k(lib):
    """A given as the transpose of a stored (K x M) matrix, B as a transpose too, with
    K split over 5 CTAs accumulating atomically."""
    M, N, K = 256, 96, 1000
    g = torch.Generator().manual_seed(3)
    At = torch.randn(K, M, generator=g).to(torch.bfloat16).cuda()  # stores A^T
    Bt = torch.randn(K, N, generator=g).to(torch.bfloat16).cuda()  # stores B^T
    C = gemm(lib, At, Bt, M, N, K, (1, M), (1, N), splits=5, bn=32)
    R = ref(At.t().contiguous(), Bt.t().contiguous())
    np.testing.assert_allclose(C.cpu().numpy(), R, rtol=1e-4, atol=1e-4 * np.sqrt(K))


def test_gemm_pipeline_long_k_ragged_edges(lib):
    """K-contiguous operands take the multi-stage cp.async pipeline: many chunks (stage
    reuse), a K tail that is not a multiple of the chunk, ragged M and N."""
    M, N, K = 301, 200, 1000 + 8
    g = torch.Generator().manual_seed(5)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    for bn, splits in ((256, 1), (64, 3)):
        C = gemm(lib, A, B, M, N, K, (K, 1), (K, 1), splits=splits, bn=bn)
        R = ref(A, B)
        np.testing.assert_allclose(C.cpu().numpy(), R, rtol=1e-4, atol=1e-4 * np.sqrt(K))


@pytest.mark.parametrize("bn", [128, 256])
def test_gemm_persistent_many_tiles(lib, bn):
    """More output tiles than SMs: each persistent CTA walks several tiles, so stage
    phases wrap many times and both TMEM accumulators alternate; ragged M and K."""
    M, N, K = 51200 + 37, 256, 320 + 24
    g = torch.Generator().manual_seed(bn)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    bias = torch.randn(N, generator=g).float().cuda()
    C = gemm(lib, A, B, M, N, K, (K, 1), (K, 1), bias, 1, bn=bn)
    R = ref(A, B, bias, 1)
    np.testing.assert_allclose(C.cpu().numpy(), R, rtol=1e-4, atol=1e-4 * np.sqrt(K))


def test_gemm_split_k_uneven(lib):
    """A split count that does not divide the K chunks (16 chunks over 7 requested
    splits); every chunk is accumulated exactly once into a pre-filled C."""
    M, N, K = 200, 64, 1024
    g = torch.Generator().manual_seed(9)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C0 = torch.randn(M, N, generator=g).float()
    C = gemm(lib, A, B, M, N, K, (K, 1), (K, 1), splits=7, bn=64, accumulate=True,
             C=C0.clone().cuda())
    R = ref(A, B) + C0.numpy().astype(np.float64)
    np.testing.assert_allclose(C.cpu().numpy(), R, rtol=1e-4, atol=1e-4 * np.sqrt(K))
