"""Mixed precision at o=30, v=300 (the size whose two forms of the (xc|bd)
block do not fit together in HBM): the solve converges, and its energy lies
within 1e-6 Eh of the FP64-class solve of the same state (the FP64-class path
is itself held to the oracle at o=4 and o=20, test_gpu_fullsize.py)."""
import pytest

pytestmark = pytest.mark.gpu


def test_c3_mixed_matches_fp64_class():
    import torch
    import synth
    import paper_2501_10515_gb300 as pkg
    o, v, h, p = 30, 300, 29, 0
    s = synth.make_system(o, v, seed=0)
    energies = {}
    for name, prec in (("mixed", pkg.ASCC_MIXED_BF16), ("fp64tc", pkg.ASCC_FP64_TC)):
        ctx = pkg.Context(o, v, s.naux, s.eps, s.B, hole=h, particle=p, linearize=1,
                          precision=prec)
        r = ctx.solve()
        torch.cuda.synchronize()
        assert r.status == 0, (name, r.status, r.iterations, r.max_resid)
        energies[name] = r.energy
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    assert abs(energies["mixed"] - energies["fp64tc"]) < 1e-6, energies
