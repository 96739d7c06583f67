"""Failure statuses and exact resume, through the C ABI.

Every failure here is made on the host (non-finite amplitudes handed in
through ascc_set_state, an iteration cap, a request larger than the server's
memory budget); nothing faults or stalls the GPU.  The checkpoint tests stop
a solve, save its iteration state (amplitudes, DIIS history, counters,
mixed-precision phase), load it into a fresh context and check that the
resumed solve ends exactly where the uninterrupted one does.
"""
import numpy as np
import pytest

import synth
from oracle import amplitudes as amp

pytestmark = pytest.mark.gpu


def _ctx(s, hole, part, **kw):
    import paper_2501_10515_gb300 as pkg
    return pkg.Context(s.o, s.v, s.naux, s.eps, s.B, hole=hole, particle=part, **kw)


def test_nonfinite_amplitudes_report_diverged():
    o, v = 4, 20
    s = synth.make_system(o, v, seed=0)
    ctx = _ctx(s, 3, 0, linearize=1)
    t1, t2, _ = amp.initial_guess(o, v, 3, 0)
    t1[0, 0] = np.nan
    ctx.set_state(t1, t2)
    res = ctx.iterate(1)
    assert res.status == 5  # ASCC_ERR_DIVERGED
    assert not np.isfinite(res.energy)
    # the context stays usable: a reset solve converges
    assert ctx.solve().status == 0


def test_iteration_cap_reports_not_converged():
    o, v = 4, 20
    s = synth.make_system(o, v, seed=0)
    ctx = _ctx(s, 3, 0, linearize=1, max_iter=2)
    res = ctx.solve()
    assert res.status == 4  # ASCC_ERR_NOT_CONVERGED
    assert res.iterations == 3  # the guess plus two updates were evaluated


def test_server_refuses_a_request_beyond_its_budget():
    import paper_2501_10515_gb300 as pkg
    from paper_2501_10515_gb300.binding import AsccError
    srv = pkg.Server(64 << 20, max_active=2)
    big = synth.make_system(12, 120, seed=1)
    with pytest.raises(AsccError) as e:
        srv.submit(big.o, big.v, big.naux, big.eps, big.B, [None])
    assert e.value.status == 2  # ASCC_ERR_OOM, nothing queued
    small = synth.make_system(2, 6, seed=2)
    srv.submit(small.o, small.v, small.naux, small.eps, small.B, [None, (1, 0)])
    srv.drain()
    res = srv.results()
    srv.close()
    assert len(res) == 2 and all(r["status"] == 0 for r in res)


@pytest.mark.parametrize("precision,triples", [(0, 0), (1, 0), (2, 1)])
def test_checkpoint_resume_reproduces_the_solve(precision, triples):
    o, v, hole, part = (4, 20, 3, 0) if not triples else (3, 9, 2, 1)
    s = synth.make_system(o, v, seed=0)
    kw = dict(linearize=1, precision=precision, triples=triples)
    ref = _ctx(s, hole, part, **kw)
    full = ref.solve()
    assert full.status == 0
    stop = max(2, full.iterations // 2)
    ref.reset()
    ref.iterate(stop)
    blob = ref.checkpoint()
    t_mid = ref.get_state()
    # a fresh context of the same state resumes from the blob
    ctx = _ctx(s, hole, part, **kw)
    ctx.restore(blob)
    for a, b in zip(ctx.get_state(), t_mid):
        assert np.array_equal(a, b)
    res = ctx.iterate(1000)
    assert res.status == 0
    assert res.iterations == full.iterations
    assert res.energy == full.energy
    # a blob of another state is refused
    other = _ctx(s, hole, part, linearize=0, precision=precision, triples=triples)
    from paper_2501_10515_gb300.binding import AsccError
    with pytest.raises(AsccError):
        other.restore(blob)


def test_bounded_wait_times_out_and_the_context_survives():
    """A bounded device wait on an mbarrier phase that nothing completes (the
    kernels' own wait function, 100 ms budget) gives up, the call reports
    ASCC_ERR_TIMEOUT, and the next tensor-core product on the same context
    runs normally."""
    import torch
    import paper_2501_10515_gb300 as pkg
    st = pkg.selftest_bounded_wait(100)
    assert st == 6, st  # ASCC_ERR_TIMEOUT
    A = torch.randn(300, 200, device="cuda", dtype=torch.float64)
    B = torch.randn(250, 200, device="cuda", dtype=torch.float64)
    C = torch.empty(300, 250, device="cuda", dtype=torch.float64)
    pkg.gemm_split_bf16(A, B, C, 3)
    torch.cuda.synchronize()
    ref = A @ B.T
    assert (C - ref).abs().max().item() < 1e-4 * ref.abs().max().item()
