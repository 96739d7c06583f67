"""Tile shapes of the split-BF16 tcgen05 GEMM and their autotuner: every
shape accumulates each output over the same K tiles in the same order, so
the three kernels, and the autotuner's pick among them, give bit-identical
products for the same split-K factor."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(1000, 700, 200), (300, 2000, 1500), (40, 900, 300),
                                   (2500, 100, 3000), (129, 257, 64)])
@pytest.mark.parametrize("level", [1, 2, 3])
def test_tile_shapes_bit_identical(M, N, K, level):
    import torch
    import paper_2501_10515_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K + level)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float64, generator=g)
    outs = []
    for tile in (1, 2, 3, -1, 0):
        for beta in (0.0, 0.5, 1.0):
            C = C0.clone()
            pkg.gemm_split_bf16(A, B, C, level, alpha=0.75, beta=beta, tile=tile)
            outs.append((tile, beta, C))
    torch.cuda.synchronize()
    # for M <= 64 < N, tile 3 and the size rules (and so the autotuner, which
    # leaves such products to the rules) exchange the operands: a second class
    exchanged = M <= 64 < N
    cls = lambda t: (t in (3, -1, 0)) if exchanged else 0
    for beta in (0.0, 0.5, 1.0):
        for c in {cls(t) for t, _, _ in outs}:
            group = [(t, C) for t, b, C in outs if b == beta and cls(t) == c]
            ref = group[0][1]
            for tile, C in group:
                assert torch.equal(C.view(torch.int64), ref.view(torch.int64)), (tile, beta)
    # and the product itself is right
    ref64 = 0.75 * (A @ B.T)
    scale = (0.75 * (A.abs() @ B.abs().T)).max().item()
    tol = {1: 1e-2, 2: 1e-4, 3: 5e-5}[level]
    assert (outs[0][2] - ref64).abs().max().item() / scale < tol


def test_autotuner_records_classes():
    import torch
    import paper_2501_10515_gb300 as pkg
    n0 = pkg.autotuned_classes()
    A = torch.randn(2048, 512, device="cuda", dtype=torch.float64)
    B = torch.randn(1536, 512, device="cuda", dtype=torch.float64)
    C = torch.empty(2048, 1536, device="cuda", dtype=torch.float64)
    pkg.gemm_split_bf16(A, B, C, 2, tile=0)
    torch.cuda.synchronize()
    n1 = pkg.autotuned_classes()
    pkg.gemm_split_bf16(A, B, C, 2, tile=0)   # the same class: no second tuning
    torch.cuda.synchronize()
    assert n1 >= max(n0, 1) and pkg.autotuned_classes() == n1
