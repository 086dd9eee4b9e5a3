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


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 128, 256)])
def test_gemm_wait_that_runs_out_reports_timeout(lib, M, N, K, monkeypatch):
    """The timeout path of the bounded mbarrier waits, made to run out without a
    fault: every stage expects 64 bytes more than its two copies deliver, so
    the copies land but no stage's barrier ever completes.  The kernel must
    give up, write SA_ETIMEOUT to the status word and leave the context usable
    (the next GEMM, without the knob, is exact).  K = 256 also makes the
    producer run out on a stage that the matrix unit never freed."""
    import torch
    from paper_2408_00018_gb300 import sa
    g = torch.Generator(device="cpu").manual_seed(11)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    D = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("SA_GEMM_TEST_STALL", "1")
    assert _gemm(lib, A, B, D, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == sa.SA_ETIMEOUT
    monkeypatch.delenv("SA_GEMM_TEST_STALL")
    status.zero_()
    assert _gemm(lib, A, B, D, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.double().cpu() @ B.double().cpu().T
    bound = K * 2.0 ** -24 * (A.double().abs().cpu() @ B.double().abs().cpu().T) + 1e-30
    assert ((D.double().cpu() - ref).abs() <= bound).all()


def test_surrogate_run_reports_gemm_timeout(lib, monkeypatch):
    """A delayed-acceptance run whose surrogate GEMMs time out reports SA_ETIMEOUT
    (the GEMMs write the run's own status word; sa_run only launches, and the
    first call that synchronises, sa_best, reports the device's status)."""
    import torch
    from paper_2408_00018_gb300 import inputs, sa
    n, C, L = 32, 256, 2
    lo, hi = inputs.box("rot_schwefel", n)
    sch = sa.Schedule(T0=10.0, rho=0.9, levels=1, sigma_frac=0.1, precision="fp32", surrogate=1)
    monkeypatch.setenv("SA_GEMM_TEST_STALL", "1")  # before sa_create, which captures the level graphs
    h = sa.create("rot_schwefel", lo, hi, n, C, L, sch, seed=3, Q=inputs.rotation(n, 1))
    h.run()
    with pytest.raises(sa.SAError) as err:
        h.best()
    assert err.value.status == sa.SA_ETIMEOUT
    monkeypatch.delenv("SA_GEMM_TEST_STALL")
    h.destroy()
    torch.cuda.synchronize()
    # the context is still usable: a fresh surrogate run completes
    h2 = sa.create("rot_schwefel", lo, hi, n, C, L, sch, seed=3, Q=inputs.rotation(n, 1))
    h2.run()
    assert np.isfinite(h2.best()[1])
    h2.destroy()
