"""The smaller hash-path CTAs split into thread groups (128 or 256 threads, each with a quarter or a
half of the CTA's run tables and its own named barrier, one block per group) against the oracle and
against whole-CTA checking (hash_groups=1).

A block goes to the smallest group whose table holds each of its runs, judged by sampling the epochs
of its records; a run may still hold more racy units than the group's pool. The library reports how
many blocks each launch group took, and the tests check that count. Cases: the grid family's 32- to
128-thread blocks (tree reductions go to groups, 2048-record transpose runs to whole CTAs) with runs
merged across missing barriers; blocks whose first run is much longer than the others (it decides
the group; one run exceeds its group's racy-unit pool and is spilled to the sort path); and a batch
mixing all of them. hash_shape=2 puts every block on the smaller shape, so small traces reach the
group launches."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import checker, diff, gpu_check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bt", [32, 64, 128])
def test_grid_family_in_thread_groups(bt):
    tr = tracegen.pattern(40 + bt, n_blocks=48, block_threads=bt, n_epochs=14, shared_units=12288,
                          global_units=1 << 20, removed_p=0.3)
    want = oracle.check(tr)
    assert diff(gpu_check(tr, path=0, hash_shape=2), want) == []
    g = checker(path=0, hash_shape=2).hash_groups()
    # tree reductions' short runs go to thread groups, 2048-record transpose runs to whole CTAs
    assert g["quarter"] + g["half"] > 0 and g["small"] > 0 and g["large"] == 0, g
    assert sum(g.values()) == tr.n_blocks
    if bt == 128:
        assert g["quarter"] == 0, g   # runs of about 950 records exceed a quarter table
    assert diff(gpu_check(tr, path=0, hash_shape=2, hash_groups=1), want) == []
    g = checker(path=0, hash_shape=2, hash_groups=1).hash_groups()
    assert g["quarter"] == g["half"] == 0 and g["small"] == tr.n_blocks, g


def _big_first_run(seed: int, distinct: int, racy: int) -> tracegen.Trace:
    """Three 64-thread blocks over 12 epochs. Block 1's epoch 0 touches `distinct` units, `racy` of them
    written by two threads (so the run holds distinct + racy records); every other run holds one record
    per thread."""
    rng = np.random.default_rng(seed)
    b = tracegen.Builder(3, 64, 4096, 1 << 12)
    for blk in range(3):
        for e in range(12):
            if blk == 1 and e == 0:
                units = rng.permutation(4096)[:distinct]
                for k, u in enumerate(units):
                    b.access(blk, k % 64, 0, int(u), tracegen.READ if k >= racy else tracegen.WRITE)
                for k in range(racy):
                    b.access(blk, (k + 1) % 64, 0, int(units[k]), tracegen.WRITE)
            else:
                for t in range(64):
                    b.access(blk, t, e, (t * 7 + e * 3) % 4096,
                             tracegen.WRITE if t % 4 == 0 else tracegen.READ, tracegen.SHARED if t % 2 else tracegen.GLOBAL)
    b.set_counts(11)
    return b.trace()


# (distinct units of block 1's first run, how many of them racy, the launch group block 1 goes to):
# runs up to 672 records never look long for a quarter table, 896 or more always do, 1792 or more
# always look long for a half table (samples every 224 records)
BIG_RUNS = [(300, 100, "quarter"), (1500, 0, "half"), (700, 700, "half"), (2500, 0, "small")]


@pytest.mark.parametrize("distinct,racy,group", BIG_RUNS)
def test_group_choice_and_hand_offs(distinct, racy, group):
    """Block 1's first run decides its launch group; 700 racy units exceed a half group's pool of 682,
    so that run is spilled to the sort path."""
    tr = _big_first_run(distinct + racy, distinct, racy)
    want = oracle.check(tr)
    assert len(want["races"]) >= racy
    assert diff(gpu_check(tr, path=0, hash_shape=2), want) == []
    g = checker(path=0, hash_shape=2).hash_groups()
    expect = {"quarter": 2, "half": 0, "small": 0, "large": 0}   # blocks 0 and 2: 64-record runs
    expect[group] += 1
    assert g == expect, g


def test_batch_with_group_and_whole_cta_blocks():
    from paper_1905_01833_gb300 import simulee
    trs = [tracegen.pattern(90 + i, n_blocks=6 + i, block_threads=(32, 64, 128, 256)[i % 4], n_epochs=5 + 3 * i,
                            shared_units=12288, global_units=1 << 18, removed_p=0.25) for i in range(8)]
    trs += [_big_first_run(7 + i, d, r) for i, (d, r, _) in enumerate(BIG_RUNS)]
    trs.append(tracegen.random_grouped(11, n_events=400))
    wants = [oracle.check(t) for t in trs]
    for groups in (0, 1):
        got = checker(path=0, hash_shape=2, hash_groups=groups).check_batch([simulee.to_device(t) for t in trs])
        for i, (g, w) in enumerate(zip(got, wants)):
            assert diff(g, w) == [], (groups, i, diff(g, w))
