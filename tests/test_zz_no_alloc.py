"""The allocation-free tensor-core GEMM entry point, through the C ABI.

ascc_gemm_split_bf16_noalloc serves callers that cannot allocate device memory
when they need the product: processes whose GPU memory was handed in full to
another pool, and code that must stay out of the CUDA allocator (which can
synchronise the device).  It must give the same product as the allocating
ascc_gemm_split_bf16 (same operand split, same K split), call after call,
with its operand planes and split-K partials in the library's fixed scratch
array.  This file is collected last on purpose.
"""
import pytest

pytestmark = pytest.mark.gpu

# the split-GEMM tolerance of tests/test_gpu_mixed.py (relative to sum |a||b|)
LEVEL_TOL = {1: 1e-2, 2: 1e-4, 3: 5e-5}


def _operands(M, N, K, seed):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float64, generator=g)
    return A, B, C0


@pytest.mark.parametrize("level", [2, 3])
def test_noalloc_matches_allocating_entry_point_twice(level):
    import torch
    import paper_2501_10515_gb300 as pkg
    for call, (M, N, K) in enumerate([(300, 500, 700), (130, 260, 1000), (64, 96, 5000)]):
        A, B, C0 = _operands(M, N, K, seed=17 + call + 10 * level)
        want = C0.clone()
        pkg.gemm_split_bf16(A, B, want, level, alpha=0.75, beta=0.5)
        got = C0.clone()
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        pkg.gemm_split_bf16_noalloc(A, B, got, level, alpha=0.75, beta=0.5)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        # same K split as the allocating call: the same FP32 partial sums
        assert (got - want).abs().max().item() <= 1e-12 * ((want.abs().max().item()) + 1.0)
        scale = (0.75 * (A.abs() @ B.abs().T)).max().item() + 1.0
        assert (got - want).abs().max().item() / scale < LEVEL_TOL[level]
        ref = 0.75 * (A @ B.T) + 0.5 * C0
        assert (got - ref).abs().max().item() / scale < LEVEL_TOL[level]


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2501_10515_gb300 as pkg
    from paper_2501_10515_gb300.binding import AsccError
    # 2 bytes * level 3 * (M + N) * K = 6 * 6000 * 1024 > 32 MiB
    A = torch.zeros(3000, 1024, device="cuda", dtype=torch.float64)
    B = torch.zeros(3000, 1024, device="cuda", dtype=torch.float64)
    C = torch.zeros(3000, 3000, device="cuda", dtype=torch.float64)
    with pytest.raises(AsccError) as e:
        pkg.gemm_split_bf16_noalloc(A, B, C, 3)
    assert e.value.status == 1
    # a request that fits still works afterwards
    A2, B2, C0 = _operands(64, 64, 64, seed=3)
    out = C0.clone()
    pkg.gemm_split_bf16_noalloc(A2, B2, out, 3, beta=1.0)
    torch.cuda.synchronize()
    assert (out - (A2 @ B2.T + C0)).abs().max().item() < 1e-3
