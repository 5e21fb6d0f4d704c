"""Dense layer on the tcgen05 tensor cores (mslice_nn_gemm_bf16) and its
operand packing (mslice_nn_pack_bf16) against FP64 products of the same
BF16-rounded operands on the CPU."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_01253_gb300 import build
    build.build()


def _bf16_round(x):
    return x.to(torch.bfloat16).to(torch.float64)


def _packed(B, x, ld):
    """[rows][ld] BF16 copy of the float32 CUDA matrix x (rows x K) through the library."""
    rows, K = x.shape
    dst = torch.empty(rows * ld, dtype=torch.bfloat16, device="cuda")
    B.mslice_nn_pack_bf16(x, x.stride(0), x.stride(1), rows, K, dst, ld)
    return dst


def test_pack_rounds_to_nearest_even_and_pads():
    from paper_2212_01253_gb300 import binding as B
    g = torch.Generator().manual_seed(3)
    x = torch.randn(70, 45, generator=g, dtype=torch.float32) * 3
    x[0, :4] = torch.tensor([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0])   # ties
    xt = x.t().contiguous().cuda()            # pack the transpose through the strides
    dst = torch.empty(70 * 48, dtype=torch.bfloat16, device="cuda")
    B.mslice_nn_pack_bf16(xt, 1, 70, 70, 45, dst, 48)
    torch.cuda.synchronize()
    got = dst.view(70, 48).cpu()
    assert torch.equal(got[:, :45], x.to(torch.bfloat16))
    assert torch.count_nonzero(got[:, 45:]) == 0


CASES = [(128, 256, 64, False, False, 0.0), (300, 520, 200, True, False, 0.0), (129, 257, 65, True, True, 0.5),
         (1, 1, 1, False, True, 0.0), (512, 768, 1024, True, True, 0.0), (64, 300, 4096, False, False, 1.0)]


@pytest.mark.parametrize("M,N,K,use_bias,relu,beta", CASES)
def test_gemm_bf16_matches_fp64_products(M, N, K, use_bias, relu, beta):
    from paper_2212_01253_gb300 import binding as B
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, generator=g)
    b = torch.randn(N, K, generator=g)
    bias = torch.randn(N, generator=g) if use_bias else None
    c0 = torch.randn(M, N, generator=g)
    lda, ldb = (K + 7) // 8 * 8, (K + 7) // 8 * 8 + 8
    A = _packed(B, a.cuda(), lda)
    Bm = _packed(B, b.cuda(), ldb)
    C = c0.clone().cuda()
    B.mslice_nn_gemm_bf16(M, N, K, A, lda, Bm, ldb, C, N, bias.cuda() if bias is not None else None, relu, beta)
    assert B.mslice_nn_gemm_bf16_status() == 0
    got = C.cpu().double()
    ref = _bf16_round(a) @ _bf16_round(b).t()
    if bias is not None:
        ref = ref + bias.double()
    if relu:
        ref = ref.clamp_min(0.0)
    ref = ref + beta * c0.double()
    # FP32 accumulation of K exact BF16 products: error within a few ulps of
    # the sum of the products' magnitudes
    scale = _bf16_round(a).abs() @ _bf16_round(b).abs().t() + beta * c0.double().abs() + 1.0
    err = (got - ref).abs() / scale
    assert float(err.max()) <= 2e-6 * np.sqrt(K) + 1e-6


def test_gemm_bf16_large_sampled_rows():
    """8192 x 8192 x 8192, 64 tiles along M and 32 along N (the throughput
    shape): 64 sampled rows against FP64 on the CPU."""
    from paper_2212_01253_gb300 import binding as B
    M = N = K = 8192
    gen = torch.Generator(device="cuda").manual_seed(5)
    a = torch.randn(M, K, generator=gen, device="cuda")
    b = torch.randn(N, K, generator=gen, device="cuda")
    A = _packed(B, a, K)
    Bm = _packed(B, b, K)
    del a, b
    C = torch.empty(M, N, device="cuda")
    B.mslice_nn_gemm_bf16(M, N, K, A, K, Bm, K, C, N)
    assert B.mslice_nn_gemm_bf16_status() == 0
    rows = torch.tensor(np.random.default_rng(1).choice(M, 64, replace=False), device="cuda")
    ar = A.view(M, K)[rows].cpu().double()
    bb = Bm.view(N, K).cpu().double()
    ref = ar @ bb.t()
    got = C[rows].cpu().double()
    scale = ar.abs() @ bb.abs().t()
    assert float(((got - ref).abs() / scale).max()) <= 2e-6 * np.sqrt(K)


def test_gemm_bf16_rejects_bad_arguments():
    from paper_2212_01253_gb300 import binding as B
    A = torch.zeros(128 * 64 + 8, dtype=torch.bfloat16, device="cuda")
    Bm = torch.zeros(256 * 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128 * 256, device="cuda")
    with pytest.raises(B.MsliceError):
        B.mslice_nn_gemm_bf16(128, 256, 64, A, 60, Bm, 64, C, 256)     # lda < K, not a multiple of 8
    with pytest.raises(B.MsliceError):
        B.mslice_nn_gemm_bf16(128, 256, 64, A, 64, Bm, 64, C, 100)     # ldc < N
    with pytest.raises(B.MsliceError):
        B.mslice_nn_gemm_bf16(128, 256, 64, A[1:], 64, Bm, 64, C, 256)  # A not 16-byte aligned
