"""Both device paths against the oracle: the hash path (traces in simulator
order: blocks one after another, epochs in order inside a block) and the
radix-sort path (forced, or taken when a trace or block does not qualify).

The hash path has its own limits and hand-offs, each exercised here: racy
units resolved in place (up to a third of a run table's entries: 2730 with
the 8192-entry table, 1365 with the 4096-entry one) or the run spilled to the
sort path (more), a run with more distinct units than its table holds (the block
falls back), epochs out of order, blocks interleaved, blocks and epochs
without records, and runs that span several 2048-record windows."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import diff, gpu_check

pytestmark = pytest.mark.gpu

PATHS = {"auto": 0, "sort": 1}
SHAPES = [1, 2]   # hash path: one 768-thread CTA per SM (8192-entry tables), two 512-thread CTAs (4096)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_grouped_random_traces(path):
    for seed in range(200):
        tr = tracegen.random_grouped(seed)
        d = diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr))
        assert d == [], f"seed {seed}: {d}"


@pytest.mark.parametrize("shape", SHAPES)
def test_grouped_random_traces_both_shapes(shape):
    for seed in range(200, 320):
        tr = tracegen.random_grouped(seed)
        d = diff(gpu_check(tr, path=0, hash_shape=shape), oracle.check(tr))
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


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nb,bt,ep,removed", [(12, 256, 32, 0.5), (3, 1024, 6, 0.3), (40, 64, 12, 0.1)])
def test_grid_family_both_shapes(shape, nb, bt, ep, removed):
    tr = tracegen.pattern(nb * 3 + ep, n_blocks=nb, block_threads=bt, n_epochs=ep, shared_units=12288,
                          global_units=1 << 20, removed_p=removed)
    assert diff(gpu_check(tr, path=0, hash_shape=shape), oracle.check(tr)) == []


def test_long_runs_and_out_of_order_epochs_fall_back():
    # 4096-record runs (single block, 256 threads x 16 accesses) span two windows of the hash path
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


def test_batch_split_between_cta_shapes():
    """A batch with at least two blocks of at most 256 threads per SM and some 1024-thread blocks:
    the first go to the two-CTA shape, the others to the one-CTA shape, in two launches over one
    block list; every trace equals checking it alone."""
    from paper_1905_01833_gb300 import simulee
    from gpu_util import checker
    trs = [tracegen.pattern(51, n_blocks=200, block_threads=64, n_epochs=6, shared_units=4096, global_units=1 << 20),
           tracegen.pattern(52, n_blocks=2, block_threads=1024, n_epochs=5, shared_units=12288, global_units=1 << 20),
           tracegen.pattern(53, n_blocks=130, block_threads=128, n_epochs=5, shared_units=4096, global_units=1 << 20),
           tracegen.pattern(54, n_blocks=3, block_threads=1024, n_epochs=4, shared_units=12288, global_units=1 << 20)]
    assert sum(t.n_blocks for t in trs if t.block_threads <= 256) >= 2 * 152
    got = checker().check_batch([simulee.to_device(t) for t in trs])
    for i, tr in enumerate(trs):
        assert diff(got[i], oracle.check(tr)) == [], f"trace {i}"


def test_batch_signature_tables_direct_and_hashed():
    """Block signatures: each trace's units in its own stretch of one direct table while all
    traces' global units together fit 2^28 slots, else a hashed (trace, unit) table (collisions
    only keep records). The same traces, declared with small and with large global spaces."""
    from paper_1905_01833_gb300 import simulee
    from gpu_util import checker
    base = [tracegen.random_grouped(900 + i, n_events=4000, n_blocks=6) for i in range(3)] + \
           [tracegen.pattern(61, n_blocks=6, block_threads=64, n_epochs=5, shared_units=4096, global_units=1 << 16)]
    for gu in (None, (1 << 27) + 5):
        trs = [t if gu is None else tracegen.Trace(t.events, t.barrier_counts, t.n_blocks, t.block_threads,
                                                   t.shared_units, gu, t.max_barriers, t.flags) for t in base]
        got = checker().check_batch([simulee.to_device(t) for t in trs])
        for i, tr in enumerate(trs):
            assert diff(got[i], oracle.check(tr)) == [], (gu, i)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_blocks_with_merged_epochs_take_the_sort_path(path):
    """Half the blocks lose a barrier, so two epochs merge into one run of two
    windows with many racy units (spilled to the sort path)."""
    tr = tracegen.pattern(21, n_blocks=16, block_threads=256, n_epochs=20, shared_units=12288,
                          global_units=1 << 20, removed_p=0.5)
    assert diff(gpu_check(tr, path=PATHS[path]), oracle.check(tr)) == []


def _racy_units_trace(k: int, n_blocks: int = 2):
    """Epoch 0: thread 0 writes units 0..k-1, thread 1 reads them (k racy units);
    epoch 1: thread 2 writes units 0..k-1 (barrier 0 needed)."""
    b = tracegen.Builder(n_blocks, 32, 4096)
    for blk in range(n_blocks):
        for u in range(k):
            b.access(blk, 0, 0, u, tracegen.WRITE)
        for u in range(k):
            b.access(blk, 1, 0, u, tracegen.READ)
        for u in range(k):
            b.access(blk, 2, 1, u, tracegen.WRITE)
    return b.set_counts(1).trace()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [1, 2, 64, 300, 1365, 1366, 2730, 2731])
def test_racy_units_in_place_and_spilled(k, shape):
    tr = _racy_units_trace(k)
    want = oracle.check(tr)
    assert len(want["races"]) == 2 * k
    assert diff(gpu_check(tr, path=0, hash_shape=shape), want) == []


@pytest.mark.parametrize("shape", SHAPES)
def test_racy_units_in_consecutive_runs(shape):
    """Racy units in every epoch, over units that overlap from run to run: each
    run resolves its racy units in the previous run's table and must leave it
    empty for the next. Run sizes (2k records) fall on both sides of the
    records held per thread (4 per thread: 2048 or 4096) and of the racy-unit
    pool (1365 or 2730)."""
    ks = [3, 700, 1, 1200, 50, 2100, 9, 1024, 1500, 2]
    b = tracegen.Builder(3, 64, 8192)
    for blk in range(3):
        for e, k in enumerate(ks):
            base = (e * 37 + blk * 11) % 4096
            for u in range(k):
                b.access(blk, (e + blk) % 5, e, base + u, tracegen.WRITE)
            for u in range(k):
                b.access(blk, 5 + (u % 3), e, base + u, tracegen.READ)
    tr = b.set_counts(len(ks) - 1).trace()
    want = oracle.check(tr)
    assert len(want["races"]) == 3 * sum(ks)
    assert diff(gpu_check(tr, path=0, hash_shape=shape), want) == []


@pytest.mark.parametrize("shape", SHAPES)
def test_run_with_more_distinct_units_than_the_table(shape):
    """One epoch of 1024 threads x 7 distinct units (7168, more than either
    table holds): the block leaves the hash path; a second block (2048
    distinct units) stays on it with the larger table."""
    rng = np.random.default_rng(4)
    b = tracegen.Builder(2, 1024, 1 << 14)
    for e in range(2):
        for k in range(7):
            for t in range(1024):
                b.access(0, t, e, (t * 7 + k + e) % (1 << 14), tracegen.WRITE if rng.random() < 0.3 else tracegen.READ)
        for t in range(1024):
            b.access(1, t, e, (t + 5 * e) % 2048, tracegen.WRITE)
    tr = b.set_counts(1).trace()
    assert diff(gpu_check(tr, path=0, hash_shape=shape), oracle.check(tr)) == []


def test_epoch_gaps_and_blocks_without_records():
    """Block 0 has records in epochs 0, 2, 5 only; block 1 has none; block 2 has
    one record; adjacency is only tested between consecutive epochs."""
    b = tracegen.Builder(3, 4, 64)
    for e in (0, 2, 5):
        for t in range(4):
            b.access(0, t, e, t if e != 2 else (t + 1) % 4, tracegen.WRITE)
    b.access(2, 3, 4, 9, tracegen.READ)
    tr = b.set_counts(6).trace()
    assert diff(gpu_check(tr, path=0), oracle.check(tr)) == []


def test_interleaved_blocks_and_late_epochs():
    """Records of two blocks alternate (the trace is not block-contiguous), and
    in a third trace one block's epochs go back (not in run order)."""
    b = tracegen.Builder(2, 8, 32)
    for i in range(64):
        b.access(i % 2, i % 8, (i // 16) % 3, i % 5, i % 3 if i % 3 != 2 else tracegen.ATOMIC)
    tr = b.set_counts(2).trace()
    assert diff(gpu_check(tr, path=0), oracle.check(tr)) == []
    b = tracegen.Builder(2, 8, 32)
    for e in (0, 1, 0, 2):
        for t in range(8):
            b.access(0, t, e, (t + e) % 8, tracegen.WRITE if t % 2 else tracegen.READ)
    for t in range(8):
        b.access(1, t, 0, t, tracegen.WRITE)
    tr = b.set_counts(2).trace()
    assert diff(gpu_check(tr, path=0), oracle.check(tr)) == []


@pytest.mark.parametrize("where", [0, 2047, 2048, 5000, -1])
def test_bad_record_inside_block_ranges(where):
    """Validation happens inside the hash path's block ranges: the first bad
    index is reported wherever it lies (window edges included)."""
    tr = tracegen.pattern(31, n_blocks=3, block_threads=256, n_epochs=6, shared_units=12288, global_units=1 << 16)
    ev = tr.events.copy()
    i = where % len(ev)
    ev[i, 3] |= np.uint32(3 << 28)   # action 3 is invalid
    ev[-1, 0] = np.uint32(1 << 20) | (ev[-1, 0] & np.uint32(0xFF))   # a later bad unit as well
    bad = tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units,
                         tr.max_barriers)
    got, want = gpu_check(bad, path=0), oracle.check(bad)
    assert diff(got, want) == []
    assert got["bad_index"] == i


@pytest.mark.parametrize("shape", SHAPES)
def test_order_checks_at_warp_and_window_edges(shape):
    """The comparison of each record with the record before it (visit order
    strictly increasing; epochs not going back inside a block) at every kind
    of position: warp starts of a run's windows (64 records apart), lanes
    either side of them, and the start of a run's second window. Runs hold
    2816 records (256 threads x 11 units), more than one window of either
    shape and fewer distinct units than the smaller table holds."""
    b = tracegen.Builder(2, 256, 4096)
    for blk in range(2):
        for e in range(4):
            for k in range(11):
                for t in range(256):
                    b.access(blk, t, e, t * 11 + k, tracegen.WRITE if (t + k + e) % 5 == 0 else tracegen.READ)
    tr = b.set_counts(3).trace()
    ev0 = tr.events
    s = 2816 * 6   # first record of run (block 1, epoch 2)
    assert ev0[s, 2] == 1 and (ev0[s, 3] >> 16) & 0xFFF == 2 and (ev0[s - 1, 3] >> 16) & 0xFFF == 1
    window = 2048 if shape == 1 else 1024
    offs = [0, 1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 127, 128, 129, 511, 512, 513]
    for p in sorted({s + o for o in offs} | {s + window + o for o in offs}):
        ev = ev0.copy()
        ev[p, 1] = ev[p - 1, 1]   # visit order repeats: the trace is invalid at p
        bad = tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                             tr.global_units, tr.max_barriers)
        got = gpu_check(bad, path=0, hash_shape=shape)
        assert (got["status"], got["bad_kind"], got["bad_index"]) == (2, 0, p), p
        if p > s:   # epoch 1 inside run 2: a valid trace whose epochs go back
            ev = ev0.copy()
            ev[p, 3] = (ev[p, 3] & ~np.uint32(0xFFF << 16)) | np.uint32(1 << 16)
            back = tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                                  tr.global_units, tr.max_barriers)
            assert diff(gpu_check(back, path=0, hash_shape=shape), oracle.check(back)) == [], p
