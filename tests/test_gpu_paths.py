"""Both device paths against the oracle: the short-interval hash path (traces
in simulator order, short (block, epoch) runs) and the radix-sort path (forced,
or taken when a trace does not qualify)."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import diff, gpu_check

pytestmark = pytest.mark.gpu

PATHS = {"auto": 0, "sort": 1}


@pytest.mark.parametrize("path", sorted(PATHS))
def test_grouped_random_traces(path):
    for seed in range(200):
        tr = tracegen.random_grouped(seed)
        d = diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr))
        assert d == [], f"seed {seed}: {d}"


@pytest.mark.parametrize("path", sorted(PATHS))
def test_grouped_wider_traces(path):
    for seed in range(6):
        tr = tracegen.random_grouped(500 + seed, n_events=20000, n_blocks=4, block_threads=128, max_epochs=8,
                                     units=64 if seed % 2 else 3000)
        d = diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr))
        assert d == [], f"seed {seed}: {d}"


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("nb,bt,ep", [(12, 256, 32), (6, 64, 9), (4, 128, 20), (2, 1024, 10)])
def test_grid_family_both_paths(path, nb, bt, ep):
    tr = tracegen.pattern(nb * 7 + ep, n_blocks=nb, block_threads=bt, n_epochs=ep, shared_units=12288,
                          global_units=1 << 20)
    assert diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr)) == []


def test_long_runs_and_out_of_order_epochs_fall_back():
    # 4096-record runs (single block, 256 threads x 16 accesses) exceed the hash path's run limit
    tr = tracegen.c1()
    assert diff(gpu_check(tr, path=0), oracle.check(tr)) == []
    # a diverged thread's accesses carry a lower epoch inside later runs: not in (block, epoch) order
    tr = tracegen.barrier(seed=3, n_blocks=20, block_threads=256, n_epochs=16, shared_units=2048, diverge_p=0.3)
    assert diff(gpu_check(tr, path=0), oracle.check(tr)) == []


def test_batch_mixing_paths():
    from paper_1905_01833_gb300 import simulee
    from gpu_util import checker
    trs = [tracegen.random_grouped(7), tracegen.random_tiny(8), tracegen.c1(),
           tracegen.pattern(3, n_blocks=5, block_threads=256, n_epochs=12, shared_units=12288, global_units=1 << 18),
           tracegen.random_grouped(9, n_events=3000), tracegen.random_tiny(10, unsorted=True)]
    got = checker().check_batch([simulee.to_device(t) for t in trs])
    for i, tr in enumerate(trs):
        assert diff(got[i], oracle.check(tr)) == [], f"trace {i}"


@pytest.mark.parametrize("path", sorted(PATHS))
def test_blocks_with_merged_epochs_take_the_sort_path(path):
    """Half the blocks lose a barrier, so two epochs merge into one run longer
    than the hash path's limit: those blocks go through the sort path, the
    rest stay on the hash path, within one trace."""
    tr = tracegen.pattern(21, n_blocks=16, block_threads=256, n_epochs=20, shared_units=12288,
                          global_units=1 << 20, removed_p=0.5)
    assert diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr)) == []
