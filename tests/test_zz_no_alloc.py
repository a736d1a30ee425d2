"""The allocation-free split GEMM, for callers that cannot call cudaMalloc
(their device memory belongs to their own allocator, or they must not pay
its implicit synchronisation): it must give what the allocating entry point
gives, on two calls in a row (the shared scratch keeps the previous call's
contents), and refuse sizes beyond its fixed scratch.  Collected last."""
import numpy as np
import pytest
import torch

import paper_1805_08990_gb300 as dme
from gpu_util import SPLIT_TOL, rel, require_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    require_gpu()
    g = torch.Generator(device="cpu").manual_seed(11)
    for M, N, K in [(200, 150, 333), (512, 384, 640)]:
        A = torch.randn(M, K, generator=g, dtype=torch.float64).cuda()
        B = torch.randn(N, K, generator=g, dtype=torch.float64).cuda()
        C_alloc = torch.empty(M, N, dtype=torch.float64, device="cuda")
        C_fixed = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        dme.dme_gemm_split(A, B, C_alloc)
        dme.dme_gemm_split_noalloc(A, B, C_fixed)
        torch.cuda.synchronize()
        a, f = C_alloc.cpu().numpy(), C_fixed.cpu().numpy()
        assert np.isfinite(f).all()
        assert rel(f, a) <= SPLIT_TOL
        assert rel(f, (A @ B.T).cpu().numpy()) < SPLIT_TOL


def test_noalloc_on_a_non_default_stream():
    """The same products enqueued on a side stream: the call waits for that
    stream itself, so the result is complete when it returns."""
    require_gpu()
    g = torch.Generator(device="cpu").manual_seed(12)
    side = torch.cuda.Stream()
    M, N, K = 300, 260, 500
    A = torch.randn(M, K, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(N, K, generator=g, dtype=torch.float64).cuda()
    C_alloc = torch.empty(M, N, dtype=torch.float64, device="cuda")
    dme.dme_gemm_split(A, B, C_alloc)
    torch.cuda.synchronize()
    side.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        C_fixed = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        side.wait_stream(torch.cuda.current_stream())
        dme.dme_gemm_split_noalloc(A, B, C_fixed, stream=side)
        f = C_fixed.cpu().numpy()
        assert np.isfinite(f).all()
        assert rel(f, C_alloc.cpu().numpy()) <= SPLIT_TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    require_gpu()
    A = torch.zeros(1024, 1024, dtype=torch.float64, device="cuda")
    C = torch.zeros(1024, 1024, dtype=torch.float64, device="cuda")
    with pytest.raises(dme.DmeError) as ei:
        dme.dme_gemm_split_noalloc(A, A, C)
    assert ei.value.status == dme.DME_EINVAL
    assert "8 MiB" in str(ei.value)
