"""Race and placement check of the T3' program (host only): every pair of
ops of a section whose memory footprints conflict must be ordered by stream
order or by an event wait.  The checker derives conflicts from the
workspace placement alone, not from the plan's own dependency lists, and a
plan without its event waits must fail it; no two intermediates may share
workspace while both are live (a collapsed placement must fail that)."""
import pytest


@pytest.mark.parametrize("o,v,naux", [(4, 20, 72), (9, 70, 237), (20, 200, 660)])
@pytest.mark.parametrize("nstreams", [1, 3, 6, 8, 16])
def test_stream_plan_is_race_free(o, v, naux, nstreams):
    import paper_2501_10515_gb300 as pkg
    assert pkg.t3p_plan_check(o, v, naux, nstreams) == 0


@pytest.mark.parametrize("nstreams", [2, 6])
def test_checker_sees_races_without_waits(nstreams):
    import paper_2501_10515_gb300 as pkg
    assert pkg.t3p_plan_check(20, 200, 660, nstreams, mode=1) > 100


@pytest.mark.parametrize("nstreams", [1, 6])
def test_checker_sees_clobbers_of_a_collapsed_placement(nstreams):
    """Every intermediate at offset 0: live tensors then share memory."""
    import paper_2501_10515_gb300 as pkg
    assert pkg.t3p_plan_check(9, 70, 237, nstreams, mode=2) > 100


def test_checker_rejects_bad_arguments():
    import paper_2501_10515_gb300 as pkg
    assert pkg.t3p_plan_check(1, 20, 72, 4) == -1
    assert pkg.t3p_plan_check(4, 20, 72, 0) == -1
