"""Mixed precision: split-BF16 tensor-core GEMM and the ASCC_MIXED_BF16 path.

The GEMM is checked against an FP64 product of the same device operands; the
mixed-precision solve is checked against the CPU oracle's FP64 solve
(energy within 1e-6 Eh per result, the bar the method's use sets).
"""
import numpy as np
import pytest

import synth
from oracle import ascc as oracle_ascc

pytestmark = pytest.mark.gpu

# relative error bars of the split levels: 8- and 16-bit operand mantissas for
# levels 1 and 2; level 3 is bounded by the FP32 accumulation of the tensor core
LEVEL_TOL = {1: 1e-2, 2: 1e-4, 3: 5e-5}


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 300, 100), (128, 256, 64), (400, 2100, 4096),
                                   (77, 5, 3000)])
@pytest.mark.parametrize("level", [1, 2, 3])
def test_split_gemm_matches_fp64(M, N, K, level):
    import torch
    import paper_2501_10515_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K + level)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float64, generator=g)
    C = C0.clone()
    pkg.gemm_split_bf16(A, B, C, level, alpha=0.5, beta=-1.0)
    torch.cuda.synchronize()
    ref = 0.5 * (A @ B.T) - C0
    err = (C - ref).abs().max().item()
    scale = (0.5 * (A.abs() @ B.abs().T)).max().item() + 1.0
    assert err / scale < LEVEL_TOL[level], (err, scale)


@pytest.mark.parametrize("level", [1, 2, 3])
@pytest.mark.parametrize("M,N,K", [(1, 1, 16), (130, 17, 200), (1000, 64, 96), (777, 65, 40),
                                   (20000, 128, 200), (300, 100, 5000), (5000, 3, 70),
                                   (17, 300, 200), (64, 1000, 3000), (1, 500, 100), (40, 129, 64)])
def test_narrow_split_gemm_matches_fp64(M, N, K, level):
    """Products with N <= 128, or M <= 64 (operands exchanged, tile stored
    transposed), run on the persistent 128 x 64 kernel: several tiles per CTA,
    ragged M, N and K, split K for K > 2048."""
    import torch
    import paper_2501_10515_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(M * 5 + N * 11 + K + level)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float64, generator=g)
    for beta in (0.0, -1.0):
        C = C0.clone()
        pkg.gemm_split_bf16(A, B, C, level, alpha=0.5, beta=beta)
        torch.cuda.synchronize()
        ref = 0.5 * (A @ B.T) + beta * C0
        scale = (0.5 * (A.abs() @ B.abs().T)).max().item() + 1.0
        assert (C - ref).abs().max().item() / scale < LEVEL_TOL[level]


@pytest.mark.parametrize("level", [1, 2, 3])
@pytest.mark.parametrize("M,N,K", [(3000, 1000, 200), (129, 257, 1024), (5000, 300, 640),
                                   (65, 4000, 96), (1000, 999, 33)])
def test_short_k_split_gemm_matches_fp64(M, N, K, level):
    """Products with a short K (at most 1024) and neither side thin run on the
    persistent kernel with 128 x 128 tiles: several tiles per CTA, ragged
    edges, both beta branches."""
    import torch
    import paper_2501_10515_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(M * 3 + N * 13 + K + level)
    A = torch.randn(M, K, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(N, K, device="cuda", dtype=torch.float64, generator=g)
    C0 = torch.randn(M, N, device="cuda", dtype=torch.float64, generator=g)
    for beta in (0.0, 0.75):
        C = C0.clone()
        pkg.gemm_split_bf16(A, B, C, level, alpha=-1.5, beta=beta)
        torch.cuda.synchronize()
        ref = -1.5 * (A @ B.T) + beta * C0
        scale = (1.5 * (A.abs() @ B.abs().T)).max().item() + 1.0
        assert (C - ref).abs().max().item() / scale < LEVEL_TOL[level]


def _rounding_cases(M, K, seed):
    """FP64 values whose FP32 rounding is decided by every kind of dropped
    tail: ties to even (both parities), just above and below a tie, carries
    into the exponent, signed zeros; exponents within 2^+-60, so that no
    plane of the split underflows."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sig = rng.integers(0, 1 << 52, size=(M, K), dtype=np.uint64)
    tail = sig & np.uint64((1 << 29) - 1)
    kind = rng.integers(0, 6, size=(M, K))
    half = np.uint64(1 << 28)
    tail = np.where(kind == 0, half, tail)                    # tie
    tail = np.where(kind == 1, half + np.uint64(1), tail)     # just above
    tail = np.where(kind == 2, half - np.uint64(1), tail)     # just below
    sig = (sig & ~np.uint64((1 << 29) - 1)) | tail
    sig = np.where(kind == 3, np.uint64((1 << 52) - 1), sig)  # carry into the exponent
    exp = rng.integers(1023 - 60, 1023 + 60, size=(M, K)).astype(np.uint64)
    neg = rng.integers(0, 2, size=(M, K)).astype(np.uint64)
    bits = (neg << np.uint64(63)) | (exp << np.uint64(52)) | sig
    x = bits.view(np.float64).copy()
    x[kind == 4] = 0.0
    x[(kind == 4) & (neg == 1)] = -0.0
    x[0, :4] = [1e18, -1e-18, 1.0, -2.0]
    return x


@pytest.mark.parametrize("M,K", [(64, 64), (64, 300), (200, 200), (130, 3000)])
def test_split_conversions_exact(M, K):
    """C = alpha A I through the split GEMM: at 3 planes the planes of an
    identity hold it exactly and every product has one nonzero term, so C is
    alpha times the FP32 rounding of A, bit for bit (power-of-two alpha: exact
    scaling; other alpha: the FP64 product); at 1 plane, the BF16 rounding of
    that FP32 value.  Covers the thin, exchanged, 128 x 128 and split-K paths."""
    import numpy as np
    import torch
    import paper_2501_10515_gb300 as pkg
    A = torch.from_numpy(_rounding_cases(M, K, M + K)).cuda()
    I = torch.eye(K, dtype=torch.float64, device="cuda")
    f32 = A.to(torch.float32)
    for level, alpha, want in ((3, -0.25, -0.25 * f32.double()), (3, 0.3, 0.3 * f32.double()),
                               (1, 2.0, 2.0 * f32.to(torch.bfloat16).double())):
        C = torch.full((M, K), np.nan, dtype=torch.float64, device="cuda")
        pkg.gemm_split_bf16(A, I, C, level, alpha=alpha, beta=0.0)
        torch.cuda.synchronize()
        same = (C.view(torch.int64) == want.view(torch.int64)) | ((C == 0) & (want == 0))
        assert bool(same.all()), (level, alpha, int((~same).sum()))


def test_split_gemm_levels_improve():
    import torch
    import paper_2501_10515_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(256, 1024, device="cuda", dtype=torch.float64, generator=g)
    B = torch.randn(512, 1024, device="cuda", dtype=torch.float64, generator=g)
    ref = A @ B.T
    errs = []
    for lev in (1, 2, 3):
        C = torch.zeros(256, 512, device="cuda", dtype=torch.float64)
        pkg.gemm_split_bf16(A, B, C, lev)
        torch.cuda.synchronize()
        errs.append((C - ref).abs().max().item())
    # level 2 gains ~2^8 over level 1; level 3 is then limited by the FP32
    # accumulation inside the tensor core, so it only has to improve on level 2
    assert errs[0] > 30 * errs[1] and errs[2] < errs[1]


def _mixed_ctx(s, hole, part, **kw):
    import paper_2501_10515_gb300 as pkg
    return pkg.Context(s.o, s.v, s.naux, s.eps, s.B, hole=hole, particle=part,
                       precision=pkg.ASCC_MIXED_BF16, **kw)


@pytest.mark.parametrize("o,v,seed,exc,lin", [(4, 20, 0, (3, 0), True), (4, 20, 0, None, False),
                                              (6, 40, 2, (5, 1), True), (6, 40, 2, (5, 1), False)])
def test_mixed_solve_matches_fp64_oracle(o, v, seed, exc, lin):
    s = synth.make_system(o, v, seed=seed)
    hole, part = exc if exc else (None, None)
    ctx = _mixed_ctx(s, hole, part, linearize=int(lin),
                     pl_hole=o - 1 if exc is None else -1, pl_particle=0 if exc is None else -1)
    res = ctx.solve()
    ref = oracle_ascc.solve_state(s.eps, s.B, o, hole, part, linearize=lin, pl_hole=o - 1,
                                  pl_particle=0)
    assert ref.converged and res.status == 0
    # the polishing phase, corrected by FP64-class residuals, lands on the FP64 fixed point
    assert abs(res.energy - ref.energy) < 1e-8, (res.energy, ref.energy)
    assert res.iterations_low > 0 and res.fp64_evaluations >= 1


def test_mixed_residual_close_to_oracle():
    o, v = 6, 40
    s = synth.make_system(o, v, seed=2)
    t1, t2, _ = synth.random_amplitudes(o, v, seed=4, scale=0.05)
    ctx = _mixed_ctx(s, 5, 2, linearize=1)
    E, r1, r2, _ = ctx.residual(t1, t2)
    hbar, Bbar, _ = oracle_ascc.prepare(s.eps, s.B, o, 5, 2)
    from oracle import spinadapted as sa
    Eo, r1o, r2o, _ = sa.residual(hbar, Bbar, o, t1, t2, linearize=True, hole=5, particle=2)
    R = np.concatenate([r1.ravel(), r2.ravel()]); Ro = np.concatenate([r1o.ravel(), r2o.ravel()])
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) < 1e-6
    assert abs(E - Eo) < 1e-7
