"""Serving: requests admitted by device footprint, run concurrently, results unchanged by the mix."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    for seed, (o, v, states) in enumerate([(4, 20, [None, (3, 0)]), (5, 30, [(4, 1)]),
                                           (6, 24, [None, (5, 0), (4, 2)]), (3, 16, [(2, 1)])]):
        s = synth.make_system(o, v, seed=seed)
        reqs.append((o, v, s, states))
    return reqs


@pytest.mark.parametrize("precision", [0, 1])
def test_results_same_alone_and_in_the_mix(precision):
    import paper_2501_10515_gb300 as pkg
    reqs = _requests()
    alone = {}
    for k, (o, v, s, states) in enumerate(reqs):
        srv = pkg.Server(8 << 30, max_active=1, precision=precision)
        srv.submit(o, v, s.naux, s.eps, s.B, states)
        srv.drain()
        for r in srv.results():
            alone[(k, r["state_index"])] = r
        srv.close()
    srv = pkg.Server(64 << 30, max_active=4, precision=precision)
    ids = [srv.submit(o, v, s.naux, s.eps, s.B, states) for (o, v, s, states) in reqs]
    srv.drain()
    mix = srv.results()
    srv.close()
    assert len(mix) == sum(len(r[3]) for r in reqs)
    workers = set()
    for r in mix:
        k = ids.index(r["request_id"])
        a = alone[(k, r["state_index"])]
        assert r["status"] == 0 and a["status"] == 0
        # deterministic kernels: bitwise equal in FP64, within 1e-6 Eh in mixed precision
        if precision == 0:
            assert r["energy"] == a["energy"]
        else:
            assert abs(r["energy"] - a["energy"]) < 1e-6
        workers.add(r["worker"])
        assert r["t_arrival"] <= r["t_start"] <= r["t_end"]
    assert len(workers) > 1


def test_admission_respects_the_memory_budget():
    import paper_2501_10515_gb300 as pkg
    from paper_2501_10515_gb300 import binding
    reqs = _requests()
    lib = binding.load()
    opt = binding.default_options()
    fps = [lib.ascc_footprint_bytes(o, v, s.naux, opt) for (o, v, s, _) in reqs]
    budget = max(fps) + min(fps) // 2       # at most one large request at a time
    srv = pkg.Server(budget, max_active=4)
    for (o, v, s, states) in reqs:
        srv.submit(o, v, s.naux, s.eps, s.B, states)
    srv.drain()
    res = srv.results()
    srv.close()
    spans = {}
    for r in res:
        a, b = spans.get(r["request_id"], (1e30, -1e30))
        spans[r["request_id"]] = (min(a, r["t_start"]), max(b, r["t_end"]))
    # at any instant the footprints of running requests fit the budget (or one runs alone)
    events = sorted({t for s in spans.values() for t in s})
    for t in events:
        running = [rid for rid, (a, b) in spans.items() if a <= t < b]
        if len(running) > 1:
            assert sum(fps[rid] for rid in running) <= budget


def test_mixed_state_that_does_not_converge_is_solved_again_fp64_class():
    """With an iteration cap too small for any state, a mixed solve ends
    NOT_CONVERGED and the server solves the state again on the FP64-class
    path: the result carries the iterations of both solves (each one the
    FP64-class context's count alone with the same cap)."""
    import paper_2501_10515_gb300 as pkg
    o, v = 4, 20
    s = synth.make_system(o, v, seed=0)
    cap = 3
    ref = pkg.Context(o, v, s.naux, s.eps, s.B, hole=3, particle=0, precision=pkg.ASCC_FP64_TC,
                      max_iter=cap)
    r_tc = ref.solve()
    ref.close()
    mix = pkg.Context(o, v, s.naux, s.eps, s.B, hole=3, particle=0,
                      precision=pkg.ASCC_MIXED_BF16, max_iter=cap)
    r_mx = mix.solve()
    mix.close()
    assert r_tc.status == 4 and r_mx.status == 4
    srv = pkg.Server(8 << 30, max_active=1, precision=pkg.ASCC_MIXED_BF16, max_iter=cap)
    srv.submit(o, v, s.naux, s.eps, s.B, [(3, 0)])
    srv.drain()
    res = srv.results()
    srv.close()
    assert len(res) == 1 and res[0]["status"] == 4
    assert res[0]["iterations"] == r_mx.iterations + r_tc.iterations
    # the server's molecule has its integrals built for mixed precision
    # (6-product split BF16), the reference context for FP64-class
    assert abs(res[0]["energy"] - r_tc.energy) < 1e-6
