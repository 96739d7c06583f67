"""Tensor-core contractions from exact BF16 digit-plane products (ASCC_FP64_TC).

The GEMM is checked against NumPy's FP64 product (a library routine, used
here as the reference of a plain matrix product), bit for bit on integer
data where the exact result is representable, and the ASCC_FP64_TC solve
and residual against the CPU oracle with the FP64 path's bars.
"""
import numpy as np
import pytest

import synth
from oracle import amplitudes as amp
from oracle import ascc as oracle_ascc
from oracle import spinadapted as sa

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gemm(A, B, alpha=1.0, beta=0.0, C0=None):
    import paper_2501_10515_gb300 as pkg
    dA = torch.tensor(A, dtype=torch.float64, device="cuda")
    dB = torch.tensor(B, dtype=torch.float64, device="cuda")
    dC = (torch.tensor(C0, dtype=torch.float64, device="cuda") if C0 is not None
          else torch.zeros(A.shape[0], B.shape[0], dtype=torch.float64, device="cuda"))
    pkg.gemm_fp64_tc(dA, dB, dC, alpha, beta)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (130, 257, 3001), (300, 140, 40), (64, 64, 5000)])
def test_digit_gemm_matches_fp64(M, N, K):
    # ragged M, N tails (not multiples of the 128 x 96 tile), K not a multiple of 32,
    # and K beyond one exact chunk of 1024
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = _gemm(A, B)
    ref = A @ B.T
    bound = np.abs(A) @ np.abs(B).T
    # 42-bit fixed point per row with the products s + t >= 6 left out: 1e-12 to 5e-12 of
    # |A||B| on Gaussian rows (a NumPy model of the format, with truncating FP32 tail sums,
    # gives 4.3e-12 on the K = 40 case)
    assert np.all(np.abs(C - ref) <= 1e-11 * bound + 1e-300)


def test_digit_gemm_alpha_beta_and_scales():
    rng = np.random.default_rng(5)
    M, N, K = 200, 150, 2100
    # rows of very different magnitude: each row keeps its own scale
    A = rng.standard_normal((M, K)) * np.logspace(-30, 30, M)[:, None]
    B = rng.standard_normal((N, K)) * np.logspace(10, -10, N)[:, None]
    C0 = rng.standard_normal((M, N))
    C = _gemm(A, B, alpha=-0.75, beta=0.5, C0=C0)
    ref = -0.75 * (A @ B.T) + 0.5 * C0
    bound = 0.75 * (np.abs(A) @ np.abs(B).T) + 0.5 * np.abs(C0)
    assert np.all(np.abs(C - ref) <= 1e-11 * bound)


def test_digit_gemm_exact_on_integers():
    # integers below 2^10 split into two digits; every kept product is exact,
    # the chunk sums are exact in FP32 and the result is an exact integer
    rng = np.random.default_rng(7)
    M, N, K = 257, 129, 4100
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(N, K)).astype(np.float64)
    C = _gemm(A, B)
    ref = (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64)
    assert np.array_equal(C, ref)


def test_digit_gemm_nan_row_and_zero_row():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((140, 300))
    B = rng.standard_normal((70, 300))
    A[3, 17] = np.nan
    A[5] = 0.0
    B[9, 4] = np.inf
    C = _gemm(A, B)
    assert np.all(np.isnan(C[3])) and np.all(np.isnan(C[:, 9]))
    assert np.all(C[5][np.arange(70) != 9] == 0.0)
    mask = np.ones_like(C, bool); mask[3] = False; mask[:, 9] = False
    assert np.all(np.isfinite(C[mask]))


def test_digit_gemm_deterministic():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((400, 3000)); B = rng.standard_normal((500, 3000))
    assert np.array_equal(_gemm(A, B), _gemm(A, B))


def _ctx(s, hole, part, **kw):
    import paper_2501_10515_gb300 as pkg
    return pkg.Context(s.o, s.v, s.naux, s.eps, s.B, hole=hole, particle=part, **kw)


@pytest.mark.parametrize("o,v,seed,exc,lin", [(4, 20, 0, (3, 0), True), (9, 70, 3, (8, 2), True),
                                             (9, 70, 3, None, True)])
def test_fp64_tc_residual_matches_oracle(o, v, seed, exc, lin):
    import paper_2501_10515_gb300 as pkg
    s = synth.make_system(o, v, seed=seed)
    hole, part = exc if exc else (None, None)
    lh, lp = exc if exc else (o - 1, 0)
    t1, t2, _ = synth.random_amplitudes(o, v, seed=seed + 100, scale=0.05)
    if exc:
        g1, g2, _ = amp.initial_guess(o, v, hole, part)
        t1 = t1 + g1; t2 = t2 + g2
    kw = dict(linearize=int(lin), pl_hole=lh if exc is None else -1,
              pl_particle=lp if exc is None else -1, precision=pkg.ASCC_FP64_TC)
    # every large contraction of the residual on the digit-plane path
    ctx = _ctx(s, hole, part, **kw)
    E, r1, r2, _ = ctx.residual(t1, t2)
    hbar, Bbar, _ = oracle_ascc.prepare(s.eps, s.B, o, hole, part)
    Eo, r1o, r2o, _ = sa.residual(hbar, Bbar, o, t1, t2, linearize=lin, hole=lh, particle=lp)
    R = np.concatenate([r1.ravel(), r2.ravel()]); Ro = np.concatenate([r1o.ravel(), r2o.ravel()])
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-9
    assert abs(E - Eo) <= 1e-10


@pytest.mark.parametrize("o,v,seed,exc", [(4, 20, 0, (3, 0)), (4, 20, 0, None),
                                          (10, 100, 0, (9, 3))])
def test_fp64_tc_solve_matches_fp64(o, v, seed, exc):
    import paper_2501_10515_gb300 as pkg
    s = synth.make_system(o, v, seed=seed)
    hole, part = exc if exc else (None, None)
    kw = dict(linearize=1, pl_hole=o - 1 if exc is None else -1,
              pl_particle=3 if exc is None else -1)
    a = _ctx(s, hole, part, precision=pkg.ASCC_FP64, **kw)
    b = _ctx(s, hole, part, precision=pkg.ASCC_FP64_TC, **kw)
    ra, rb = a.solve(), b.solve()
    assert ra.status == 0 and rb.status == 0
    assert abs(ra.energy - rb.energy) <= 1e-10
    # the accepted amplitudes satisfy the FP64 equations
    t1, t2, _ = b.get_state()
    _, r1, r2, _ = a.residual(t1, t2)
    assert max(np.abs(r1).max(), np.abs(r2).max()) <= 2e-8
