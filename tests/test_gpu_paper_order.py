"""The paper's visit-order counters (flag PAPER_ORDER) on the device, against the oracle.

The device builds each global record's visit order (its block's earlier
epochs touching the unit) by a segmented scan of the sorted global stream,
keys the inter-block elements by it, and judges barriers against a unit's next
non-empty epoch. Every case here is compared with the oracle record for
record: the hand-built pins, random traces (tiny, grouped, unsorted), the grid
family at sizes that span many scan tiles, and a batch that mixes flagged and
unflagged traces (whose inter-block keys then carry an empty order field).
"""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import diff, gpu_check

pytestmark = pytest.mark.gpu


def _paper(tr):
    return tracegen.Trace(tr.events, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                          tr.global_units, tr.max_barriers, tr.flags | tracegen.PAPER_ORDER)


def test_pins():
    import test_oracle_paper_order as pins
    for name, (rows, nb, counts, *_rest) in pins.CASES.items():
        tr = pins._trace(rows, n_blocks=nb, counts=counts)
        assert diff(gpu_check(tr), oracle.check(tr)) == [], name


@pytest.mark.parametrize("chunk", range(3))
def test_tiny_random(chunk):
    for seed in range(chunk * 100, chunk * 100 + 100):
        tr = _paper(tracegen.random_tiny(seed, unsorted=(seed % 5 == 2)))
        assert diff(gpu_check(tr), oracle.check(tr)) == [], seed


def test_grouped_random():
    for seed in range(60):
        tr = _paper(tracegen.random_grouped(700 + seed))
        assert diff(gpu_check(tr), oracle.check(tr)) == [], seed


@pytest.mark.parametrize("nb,bt,ep,removed", [(12, 256, 32, 0.1), (40, 64, 12, 0.5), (3, 1024, 6, 0.3)])
def test_grid_family(nb, bt, ep, removed):
    tr = _paper(tracegen.pattern(nb * 5 + ep, n_blocks=nb, block_threads=bt, n_epochs=ep, shared_units=12288,
                                 global_units=1 << 20, removed_p=removed))
    want = oracle.check(tr)
    assert diff(gpu_check(tr), want) == []
    # the flag changes the answer on these traces (inter-block groups split by visit order)
    plain = oracle.check(tracegen.pattern(nb * 5 + ep, n_blocks=nb, block_threads=bt, n_epochs=ep,
                                          shared_units=12288, global_units=1 << 20, removed_p=removed))
    assert plain["races"].tobytes() != want["races"].tobytes()


def test_gaps_in_every_unit():
    """Every unit is touched every other epoch only, by rotating threads: each barrier's verdict
    depends on the next non-empty epoch of the units."""
    rng = np.random.default_rng(9)
    b = tracegen.Builder(6, 64, 256, 256)
    for blk in range(6):
        for e in range(10):
            for u in range(e % 2, 256, 2):
                if rng.random() < 0.3:
                    act = int(rng.choice([tracegen.READ, tracegen.WRITE, tracegen.ATOMIC]))
                    b.access(blk, int((u + e * 7 + blk) % 64), e, u, act,
                             tracegen.GLOBAL if u % 3 == 0 else tracegen.SHARED)
    tr = _paper(b.set_counts(9).trace())
    assert diff(gpu_check(tr), oracle.check(tr)) == []


def test_batch_mixing_flagged_and_plain():
    from paper_1905_01833_gb300 import simulee
    from gpu_util import checker
    base = [tracegen.pattern(3, n_blocks=5, block_threads=256, n_epochs=12, shared_units=12288, global_units=1 << 18),
            tracegen.random_grouped(9, n_events=3000), tracegen.random_tiny(10, unsorted=True), tracegen.c1()]
    trs = [base[0], _paper(base[0]), base[1], _paper(base[1]), _paper(base[2]), base[3]]
    got = checker().check_batch([simulee.to_device(t) for t in trs])
    for i, tr in enumerate(trs):
        assert diff(got[i], oracle.check(tr)) == [], f"trace {i}"


def test_flag_rules():
    """Not combinable with statement words (EINVAL before any launch)."""
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.with_statements(tracegen.random_tiny(1), seed=1)
    tr.flags |= tracegen.PAPER_ORDER
    with pytest.raises(RuntimeError):
        gpu_check(tr)
