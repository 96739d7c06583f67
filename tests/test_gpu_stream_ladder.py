"""The streamed particle-particle ladder (ascc_options.ladder_stream = 1).

The bare (xc|bd) block is rebuilt in x-chunks inside every residual instead
of being stored; the chunk size is forced down to 1 MB here so that every
orbital x is a chunk of its own and the occupied/virtual chunk boundaries and
the column offsets of each chunk are all exercised.  Results must meet the
same bars against the CPU oracle as the stored block.
"""
import numpy as np
import pytest

import synth
from oracle import amplitudes as amp
from oracle import ascc as oracle_ascc
from oracle import spinadapted as sa

pytestmark = pytest.mark.gpu

# precision -> (relative residual norm, energy) bars of the stored-block tests
BARS = {"ASCC_FP64": (1e-9, 1e-10), "ASCC_FP64_TC": (1e-9, 1e-10), "ASCC_MIXED_BF16": (5e-6, 1e-8)}


@pytest.fixture(autouse=True)
def small_chunks(monkeypatch):
    monkeypatch.setenv("ASCC_LADDER_CHUNK_MB", "1")


@pytest.mark.parametrize("prec", sorted(BARS))
@pytest.mark.parametrize("exc", [(8, 2), None])
def test_streamed_residual_matches_oracle(prec, exc):
    import paper_2501_10515_gb300 as pkg
    o, v, seed = 9, 70, 3
    s = synth.make_system(o, v, seed=seed)
    hole, part = exc if exc else (None, None)
    lh, lp = exc if exc else (o - 1, 0)
    t1, t2, _ = synth.random_amplitudes(o, v, seed=seed + 100, scale=0.05)
    if exc:
        g1, g2, _ = amp.initial_guess(o, v, hole, part)
        t1 = t1 + g1; t2 = t2 + g2
    ctx = pkg.Context(o, v, s.naux, s.eps, s.B, hole=hole, particle=part, linearize=1,
                      pl_hole=-1 if exc else lh, pl_particle=-1 if exc else lp,
                      precision=getattr(pkg, prec), ladder_stream=1)
    E, r1, r2, _ = ctx.residual(t1, t2)
    ctx.close()
    hbar, Bbar, _ = oracle_ascc.prepare(s.eps, s.B, o, hole, part)
    Eo, r1o, r2o, _ = sa.residual(hbar, Bbar, o, t1, t2, linearize=True, hole=lh, particle=lp)
    R = np.concatenate([r1.ravel(), r2.ravel()]); Ro = np.concatenate([r1o.ravel(), r2o.ravel()])
    rtol, etol = BARS[prec]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= rtol
    assert abs(E - Eo) <= etol


def test_streamed_mixed_solve_matches_stored():
    import paper_2501_10515_gb300 as pkg
    o, v = 4, 20
    s = synth.make_system(o, v, seed=0)
    kw = dict(hole=3, particle=0, linearize=1, precision=pkg.ASCC_MIXED_BF16)
    a = pkg.Context(o, v, s.naux, s.eps, s.B, ladder_stream=-1, **kw)
    b = pkg.Context(o, v, s.naux, s.eps, s.B, ladder_stream=1, **kw)
    ra, rb = a.solve(), b.solve()
    a.close(); b.close()
    assert ra.status == 0 and rb.status == 0
    assert abs(ra.energy - rb.energy) <= 1e-9
