"""The tcgen05 BF16 GEMM (sa_gemm_bf16) against an FP64 reference.

BF16 x BF16 products are exact in FP32; only the FP32 accumulation rounds, so
|D - A B^T| <= K u32 (|A| |B|^T) elementwise (u32 = 2^-24), checked per element.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_00018_gb300 import sa
    return sa.load()


def _gemm(lib, A, B, D, status):
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    M, K = A.shape
    N = B.shape[0]
    return lib.sa_gemm_bf16(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()), B.stride(0),
                            ctypes.c_void_p(D.data_ptr()), D.stride(0), M, N, K, ctypes.c_void_p(status.data_ptr()), s)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 64), (256, 128, 128), (384, 192, 512),
                                   (512, 512, 1024), (1024, 256, 320)])
def test_gemm_matches_fp64_reference(lib, M, N, K):
    import torch
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _gemm(lib, A, B, D, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.double().cpu() @ B.double().cpu().T
    bound = K * 2.0 ** -24 * (A.double().abs().cpu() @ B.double().abs().cpu().T) + 1e-30
    err = (D.double().cpu() - ref).abs()
    assert torch.isfinite(D).all()
    assert (err <= bound).all(), float((err / bound).max())


def test_gemm_strided_operands_and_bad_shapes(lib):
    import torch
    g = torch.Generator(device="cpu").manual_seed(5)
    Aw = torch.randn(256, 192, generator=g).to(torch.bfloat16).cuda()
    Bw = torch.randn(128, 256, generator=g).to(torch.bfloat16).cuda()
    A, B = Aw[:, :128], Bw[:, 64:192]  # leading dimensions 192 and 256
    Dw = torch.zeros(256, 160, dtype=torch.float32, device="cuda")
    D = Dw[:, :128]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _gemm(lib, A, B, D, status) == 0
    torch.cuda.synchronize()
    ref = A.double().cpu() @ B.double().cpu().T
    assert (D.double().cpu() - ref).abs().max() <= 128 * 2.0 ** -24 * (A.double().abs().cpu() @ B.double().abs().cpu().T).max()
    assert (Dw[:, 128:] == 0).all()  # nothing written outside D
    from paper_2408_00018_gb300 import sa
    bad = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    assert _gemm(lib, bad, B, D, status) == sa.SA_EINVAL
