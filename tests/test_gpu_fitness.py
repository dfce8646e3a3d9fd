"""GPU parity of the Eq. 1 fitness (simulee_fitness_batch) against the oracle.

Integer sums and ranges: the tolerance is zero. Every field of every trace's
result is compared, for single traces and batches (each trace's result must
equal the oracle's for that trace alone), valid and bad traces, sorted and
unsorted, empty ones, and key widths that need 64-bit keys.

The library counts traces whose blocks are contiguous in record order and hold
at least 1024 records on average with one read per block (a table per CTA, a
bitmap of global units; the grid-family traces here) and sends to its
radix sort the records of a block with more distinct (unit, thread) pairs than
that table takes (49,152 entries at most) and every record of a trace whose blocks are
not contiguous (the unsorted random traces); both hand-offs are tested here,
alone and mixed in one batch.
"""
import numpy as np
import pytest

import oracle
import tracegen
import cases

pytestmark = pytest.mark.gpu

FIELDS = ("status", "bad_kind", "bad_index", "n_addresses", "n_pairs", "shared_lo", "shared_hi", "global_lo",
          "global_hi")


def _checker():
    from gpu_util import checker
    return checker()


def _gpu(trs):
    from paper_1905_01833_gb300 import simulee
    return _checker().fitness_batch([simulee.to_device(t) for t in trs])


def _diff(got, want):
    return [f"{k}: gpu {got[k]} oracle {want[k]}" for k in FIELDS if int(got[k]) != int(want[k])]


@pytest.mark.parametrize("chunk", range(3))
def test_random_traces_one_by_one(chunk):
    for seed in range(chunk * 60, chunk * 60 + 60):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 4 == 1))
        d = _diff(_gpu([tr])[0], oracle.fitness(tr))
        assert d == [], f"seed {seed}: {d}"


def test_random_batch_equals_each_alone():
    trs = [tracegen.random_tiny(7000 + i, unsorted=(i % 3 == 0)) for i in range(150)]
    got = _gpu(trs)
    for i, tr in enumerate(trs):
        assert _diff(got[i], oracle.fitness(tr)) == [], f"trace {i}"


@pytest.mark.parametrize("nb,bt,ep", [(6, 64, 9), (4, 256, 12), (2, 1024, 6)])
def test_grid_family(nb, bt, ep):
    tr = tracegen.pattern(nb + ep, n_blocks=nb, block_threads=bt, n_epochs=ep, shared_units=12288,
                          global_units=1 << 20)
    assert _diff(_gpu([tr])[0], oracle.fitness(tr)) == []


def test_strided_and_barrier_families_in_one_batch():
    trs = [tracegen.c1(), tracegen.barrier(seed=5, n_blocks=6, block_threads=256, n_epochs=12, shared_units=2048,
                                           diverge_p=0.2), tracegen.random_grouped(3)]
    got = _gpu(trs)
    for i, tr in enumerate(trs):
        assert _diff(got[i], oracle.fitness(tr)) == [], f"trace {i}"


def test_bad_and_empty_traces_in_a_batch():
    trs = []
    for what, idx in cases.BAD_RECORDS:
        trs.append(cases.bad_record(what, idx)[0])
    trs.append(cases.bad_count()[0])
    trs.append(tracegen.Builder(2, 4, 8, 8).set_counts(0).trace())
    trs.append(tracegen.random_tiny(11))
    got = _gpu(trs)
    for i, tr in enumerate(trs):
        assert _diff(got[i], oracle.fitness(tr)) == [], f"trace {i}"


def test_wide_keys():
    """Many blocks x many threads and a large global space: keys wider than 32 bits."""
    tr = tracegen.random_tiny(99, n_events=50000, n_blocks=3000, block_threads=300, max_epochs=3, units=1 << 30)
    got = _gpu([tr])[0]
    assert _diff(got, oracle.fitness(tr)) == []


def test_full_size_grid_workload():
    """The 61M-record grid workload: fitness against the oracle on the same trace."""
    tr = tracegen.c2()
    got = _gpu([tr])[0]
    want = oracle.fitness(tr)
    assert _diff(got, want) == []
    assert 0 < got["n_addresses"] <= got["n_pairs"]


def _one_big_block(seed: int) -> tracegen.Trace:
    """Three 1024-thread blocks in record order; block 1 makes 64 distinct shared-unit pairs and 8 global-unit
    pairs per thread (73,728 pairs, more than a block table takes), shared with its neighbours' units."""
    rng = np.random.default_rng(seed)
    rows = []
    for b in range(3):
        per = 72 if b == 1 else 3
        for k in range(per):
            t = np.arange(1024)
            glob = k % 9 == 8
            unit = (t * 64 + k + rng.integers(0, 3)) % (1 << 16) if not glob else (b * 7919 + t * 8 + k) % (1 << 18)
            rows.append((unit, b, t, 0, rng.integers(0, 3, size=1024), 1 if glob else 0))
    u = np.concatenate([r[0] for r in rows])
    blk = np.concatenate([np.full(1024, r[1]) for r in rows])
    tid = np.concatenate([r[2] for r in rows])
    act = np.concatenate([r[4] for r in rows])
    sp = np.concatenate([np.full(1024, r[5]) for r in rows])
    ev = tracegen.pack(u, np.arange(len(u)), blk, tid, 0, act, sp)
    return tracegen.Trace(ev, np.zeros(3 * 1024, dtype=np.uint32), 3, 1024, 1 << 16, 1 << 18, 0)


def test_block_with_more_pairs_than_its_table():
    tr = _one_big_block(3)
    want = oracle.fitness(tr)
    assert want["n_pairs"] > 49152
    assert _diff(_gpu([tr])[0], want) == []


def test_batch_mixing_single_read_and_sorted_traces():
    trs = [_one_big_block(4), tracegen.random_tiny(31, unsorted=True), tracegen.random_grouped(32, n_events=3000),
           tracegen.pattern(9, n_blocks=5, block_threads=256, n_epochs=10, shared_units=12288, global_units=1 << 20),
           cases.bad_count()[0], tracegen.random_tiny(33, n_events=2000, n_blocks=7)]
    got = _gpu(trs)
    for i, tr in enumerate(trs):
        assert _diff(got[i], oracle.fitness(tr)) == [], f"trace {i}"



def test_blocks_out_of_order_fall_back_to_the_sort():
    """Large blocks whose records come block by block but not in block order: the single read finds a record
    of another block in a block's range and the whole trace is counted from sorted keys."""
    tr = tracegen.pattern(12, n_blocks=6, block_threads=256, n_epochs=8, shared_units=12288, global_units=1 << 20)
    ev = tr.events
    order = np.concatenate([np.nonzero(ev[:, 2] == b)[0] for b in (3, 1, 0, 5, 2, 4)])
    ev = np.ascontiguousarray(ev[order])
    ev[:, 1] = np.arange(len(ev), dtype=np.uint32)   # visit orders in the new record order
    tr2 = tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units,
                         tr.max_barriers)
    want = oracle.fitness(tr2)
    assert want["n_addresses"] == oracle.fitness(tr)["n_addresses"]
    assert _diff(_gpu([tr2])[0], want) == []
