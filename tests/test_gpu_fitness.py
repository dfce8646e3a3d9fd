"""GPU parity of the Eq. 1 fitness (simulee_fitness_batch) against the oracle.

Integer sums and ranges: the tolerance is zero. Every field of every trace's
result is compared, for single traces and batches (each trace's result must
equal the oracle's for that trace alone), valid and bad traces, sorted and
unsorted, empty ones, and key widths that need 64-bit keys.
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
