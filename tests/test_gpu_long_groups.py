"""Hot units: groups of the segmented reduction that span many of its 2048-element tiles (a global constant
read by every thread of the grid, broadcast shared reads of 1024-thread blocks on the sort path), with races
and barrier adjacency inside and across them. Every result equals the oracle's."""
import pytest

import oracle
import tracegen
from gpu_util import diff, gpu_check

CASES = {
    # one inter-block group of 64 x 256 x 8 global reads: 64 tiles, finished by one look-back
    "grid_constant": dict(n_blocks=64),
    # a group of 1M elements: 512 tiles, a look-back of several 256-tile steps
    "grid_constant_long": dict(n_blocks=256, n_epochs=16),
    # intra-block groups of 12 x 1024 reads (six tiles each) with writes and adjacency across tiles
    "shared_broadcast": dict(n_blocks=4, block_threads=1024, n_epochs=6, reads=12, global_const=False),
    "read_only_constant": dict(n_blocks=96, writers=False),
}


@pytest.mark.gpu
@pytest.mark.parametrize("path", [0, 1], ids=["auto", "sort"])
@pytest.mark.parametrize("name", list(CASES))
def test_hot_unit_groups_equal_oracle(name, path):
    tr = tracegen.broadcast(**CASES[name])
    assert diff(gpu_check(tr, path=path), oracle.check(tr)) == []


@pytest.mark.gpu
@pytest.mark.parametrize("marks", [0, 2], ids=["once_per_run_of_lanes", "every_record"])
def test_signature_marks_of_hot_units(marks):
    """Marking a global unit's block signature once per run of lanes that hold it, or once per record,
    gives the same results."""
    tr = tracegen.broadcast(n_blocks=48, block_threads=256, n_epochs=6, reads=2)
    assert diff(gpu_check(tr, hot_unit_marks=marks), oracle.check(tr)) == []


@pytest.mark.gpu
@pytest.mark.parametrize("ctas", [1, 2, 4])
def test_reduction_grid_sizes(ctas):
    """The look-back holds for any number of CTAs per SM (tiles are claimed in order)."""
    tr = tracegen.broadcast(n_blocks=32, block_threads=512, n_epochs=8, reads=6)
    assert diff(gpu_check(tr, path=1, reduce_ctas_per_sm=ctas), oracle.check(tr)) == []


@pytest.mark.gpu
def test_hot_units_with_the_paper_counters_and_warp_rules():
    tr = tracegen.broadcast(n_blocks=16, block_threads=256, n_epochs=8, reads=4)
    tr.flags |= tracegen.PAPER_ORDER
    assert diff(gpu_check(tr), oracle.check(tr)) == []
    tw = tracegen.with_statements(tracegen.broadcast(n_blocks=8, block_threads=256, n_epochs=6, reads=2))
    assert diff(gpu_check(tw), oracle.check(tw)) == []


@pytest.mark.gpu
def test_hot_units_in_a_batch():
    """Groups of several traces side by side in one stream: a long group ends where the next trace's begins."""
    from paper_1905_01833_gb300 import simulee
    trs = [tracegen.broadcast(n_blocks=40), tracegen.c1(), tracegen.broadcast(7, n_blocks=8, block_threads=1024,
                                                                             n_epochs=4, reads=3),
           tracegen.random_grouped(5, n_events=700)]
    got = simulee.Checker(0).check_batch([simulee.to_device(t) for t in trs])
    for i, t in enumerate(trs):
        assert diff(got[i], oracle.check(t)) == [], f"trace {i}"
