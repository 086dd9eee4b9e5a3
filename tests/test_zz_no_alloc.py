"""The non-allocating argmin entry point (sa_argmin_f64_static).

It serves callers that cannot allocate device memory (a host framework that
owns the device's memory, latency-critical loops where cudaMalloc would
synchronise the device).  Its result must equal the allocating entry point's
(sa_argmin_f64) exactly, call after call, since both reduce the same values
with the same lowest-index rule.  This file is collected last on purpose.
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


def _call_both(lib, F):
    import torch
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    count = F.numel()
    scratch = torch.empty(max(1, lib.sa_argmin_scratch_bytes(count)), dtype=torch.uint8, device="cuda")
    i1 = torch.full((), -7, dtype=torch.int64, device="cuda")
    v1 = torch.full((), -7.0, dtype=torch.float64, device="cuda")
    i2 = torch.full((), -7, dtype=torch.int64, device="cuda")
    v2 = torch.full((), -7.0, dtype=torch.float64, device="cuda")
    assert lib.sa_argmin_f64(ctypes.c_void_p(F.data_ptr()), count, ctypes.c_void_p(i1.data_ptr()),
                             ctypes.c_void_p(v1.data_ptr()), ctypes.c_void_p(scratch.data_ptr()), s) == 0
    assert lib.sa_argmin_f64_static(ctypes.c_void_p(F.data_ptr()), count, ctypes.c_void_p(i2.data_ptr()),
                                    ctypes.c_void_p(v2.data_ptr()), s) == 0
    torch.cuda.synchronize()
    return (int(i1.item()), float(v1.item())), (int(i2.item()), float(v2.item()))


def test_static_scratch_argmin_equals_allocating_argmin(lib):
    import torch
    rng = np.random.default_rng(5)
    for count in (1, 2049, 1_000_003, 4_194_304):
        for call in range(2):  # two calls in a row share the scratch
            F = np.round(rng.standard_normal(count), 2)
            if count > 100:
                F[rng.integers(0, count, 50)] = np.nan
            d = torch.tensor(F, device="cuda")
            (a_i, a_v), (b_i, b_v) = _call_both(lib, d)
            assert b_i == a_i and (b_v == a_v), (count, call)
            exp = int(np.argmin(np.where(np.isnan(F), np.inf, F)))
            assert b_i == exp


def test_static_scratch_rejects_too_large_and_null(lib):
    import torch
    from paper_2408_00018_gb300 import sa
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros((), dtype=torch.int64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many = sa.ARGMIN_STATIC_MAX_COUNT + 1
    assert lib.sa_argmin_f64_static(ctypes.c_void_p(d.data_ptr()), too_many, ctypes.c_void_p(idx.data_ptr()),
                                    ctypes.c_void_p(d.data_ptr()), s) == sa.SA_EINVAL
    assert lib.sa_argmin_f64_static(None, 4, None, None, s) == sa.SA_EINVAL


def test_static_scratch_at_its_maximum_count(lib):
    """The largest count the fixed array serves (2^27 doubles, 65 536 partials):
    the minimum sits in the last 2048-input span, so the last partial slot of
    the array decides the result; two calls in a row, the second with the
    minimum moved, check that stale partials never leak into a result."""
    import torch
    from paper_2408_00018_gb300 import sa
    count = sa.ARGMIN_STATIC_MAX_COUNT
    F = torch.ones(count, dtype=torch.float64, device="cuda")
    for pos in (count - 1, count - 2048):
        F.fill_(1.0)
        F[pos] = -3.0
        F[pos - 1] = -3.0 if pos == count - 2048 else 1.0  # a tie across the last span boundary
        (a_i, a_v), (b_i, b_v) = _call_both(lib, F)
        exp = pos - 1 if pos == count - 2048 else pos
        assert (a_i, a_v) == (exp, -3.0)
        assert (b_i, b_v) == (a_i, a_v)
    del F
    torch.cuda.empty_cache()
