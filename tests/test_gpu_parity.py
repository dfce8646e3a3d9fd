"""GPU parity: the CUDA path through the C ABI against the CPU oracle, byte for byte.

All results are integers, so the tolerance is zero: every field of every
output record, every count, the status and the first bad index must match.
"""
import numpy as np
import pytest

import oracle
import tracegen
import cases
import golden_io
from gpu_util import checker, diff, gpu_check

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("chunk", range(4))
def test_tiny_random_traces(chunk):
    for seed in range(chunk * 150, chunk * 150 + 150):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 5 == 2))
        d = diff(gpu_check(tr), oracle.check(tr))
        assert d == [], f"seed {seed}: {d}"


@pytest.mark.parametrize("seed", range(6))
def test_wide_random_traces(seed):
    """Bigger random traces: many tiles per sort pass and long groups that span tiles."""
    tr = tracegen.random_tiny(1000 + seed, n_events=40000, n_blocks=3 + seed, block_threads=64, max_epochs=6,
                              units=40 if seed % 2 else 5000, unsorted=(seed == 5))
    d = diff(gpu_check(tr), oracle.check(tr))
    assert d == [], d


@pytest.mark.parametrize("name", sorted(cases.ALL))
def test_closed_form_cases(name):
    tr, exp = cases.ALL[name]()
    got = gpu_check(tr)
    assert cases.check_expect(got, exp) == []
    assert diff(got, oracle.check(tr)) == []


def test_golden_examples():
    for name in ("fig8_memory_unit.txt", "kaldi_copy_from_mat.txt"):
        for tr, exp in golden_io.load(name):
            got = gpu_check(tr)
            assert golden_io.race_tuples(got) == exp["races"]
            assert diff(got, oracle.check(tr)) == []


@pytest.mark.parametrize("what,idx", cases.BAD_RECORDS)
def test_bad_records(what, idx):
    tr, want = cases.bad_record(what, idx)
    got = gpu_check(tr)
    assert (got["status"], got["bad_kind"], got["bad_index"]) == want
    assert got["n_races"] == 0 and len(got["races"]) == 0


def test_bad_counts_before_records():
    tr, want = cases.bad_count()
    got = gpu_check(tr)
    assert (got["status"], got["bad_kind"], got["bad_index"]) == want


def test_bad_record_in_a_large_trace():
    tr = tracegen.pattern(3, n_blocks=40, block_threads=128, n_epochs=12, shared_units=4096, global_units=1 << 18)
    for idx in (tr.n_events - 1, tr.n_events // 2 + 12345, 4097):
        t2 = tracegen.Trace(tr.events.copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                            tr.global_units, tr.max_barriers)
        t2.events[idx, 1] = t2.events[idx - 1, 1]
        got = gpu_check(t2)
        assert (got["status"], got["bad_kind"], got["bad_index"]) == (2, 0, idx)


def test_strided_single_block():
    tr = tracegen.c1()
    assert diff(gpu_check(tr), oracle.check(tr)) == []


@pytest.mark.parametrize("nb,bt,ep", [(16, 256, 32), (5, 64, 9), (3, 1024, 12), (64, 128, 20)])
def test_grid_pattern(nb, bt, ep):
    tr = tracegen.pattern(nb + bt + ep, n_blocks=nb, block_threads=bt, n_epochs=ep, shared_units=12288,
                          global_units=1 << 20)
    assert diff(gpu_check(tr), oracle.check(tr)) == []


def test_barrier_family():
    tr = tracegen.barrier(seed=5, n_blocks=40, block_threads=256, n_epochs=24, shared_units=2048, diverge_p=0.1,
                          redirect_p=1e-4)
    got = gpu_check(tr)
    assert diff(got, oracle.check(tr)) == []
    assert [int(b) for b in got["divergence"]["block"]] == list(tr.meta["divergent_blocks"])


@pytest.mark.parametrize("seed", [1, 2])
def test_unsorted_permutation(seed):
    tr = tracegen.pattern(seed, n_blocks=6, block_threads=64, n_epochs=10, shared_units=2048, global_units=1 << 15)
    base = gpu_check(tr)
    perm = np.random.default_rng(seed).permutation(tr.n_events)
    tr2 = tracegen.Trace(tr.events[perm].copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                         tr.shared_units, tr.global_units, tr.max_barriers, tracegen.UNSORTED)
    got = gpu_check(tr2)
    assert diff(got, base) == []
    assert diff(got, oracle.check(tr2)) == []


def test_empty_and_degenerate():
    b = tracegen.Builder(3, 5, 4, 4)
    b.set_counts(2)
    tr = b.trace()
    assert diff(gpu_check(tr), oracle.check(tr)) == []
    # one unit hit by every record: a single group spanning many sort tiles
    n = 30000
    rng = np.random.default_rng(0)
    ev = tracegen.pack(0, np.arange(n), rng.integers(0, 4, n), rng.integers(0, 32, n), 0,
                       rng.choice([0, 1, 2], n, p=[0.9, 0.02, 0.08]), 1)
    tr = tracegen.Trace(ev, np.zeros(4 * 32, np.uint32), 4, 32, 1, 1, 0)
    assert diff(gpu_check(tr), oracle.check(tr)) == []


def test_truncation_keeps_canonical_prefix():
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.c1()
    want = oracle.check(tr)
    chk = checker()
    got = chk.check(simulee.to_device(tr), races_cap=100, red_cap=0, grid_cap=0)
    assert got["status"] == simulee.ETRUNC
    assert got["n_races"] == len(want["races"])
    assert np.array_equal(got["races"], want["races"][:100])


def test_single_output_entry_points():
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.barrier(seed=9, n_blocks=20, block_threads=128, n_epochs=16, shared_units=1024, diverge_p=0.2)
    want = oracle.check(tr)
    dt = simulee.to_device(tr)
    chk = checker()
    r = chk.check_races(dt)
    assert r["status"] == 0 and np.array_equal(r["races"], want["races"])
    d = chk.check_divergence(dt)
    assert d["status"] == 0 and np.array_equal(d["divergence"], want["divergence"])
    b = chk.check_redundant_barriers(dt)
    assert b["status"] == 0 and np.array_equal(b["redundant"], want["redundant"])
    assert np.array_equal(b["grid_redundant"], want["grid_redundant"])


def test_repeatable_and_deterministic():
    tr = tracegen.pattern(11, n_blocks=32, block_threads=256, n_epochs=16, shared_units=12288, global_units=1 << 20)
    a = gpu_check(tr)
    b = gpu_check(tr)
    for k in ("races", "divergence", "redundant", "grid_redundant"):
        assert a[k].tobytes() == b[k].tobytes()


def test_bounded_wait_reports_timeout_and_context_survives():
    """A sort tile that never publishes its counts: the next tile's wait is
    bounded, the call reports ETIMEOUT, and the next call on the GPU is fine."""
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.pattern(2, n_blocks=16, block_threads=256, n_epochs=16, shared_units=12288, global_units=1 << 20)
    stalled = simulee.Checker(0, wait_limit_us=20000, test_withhold=3, path=1)   # sort path: long radix passes
    got = stalled.check(simulee.to_device(tr))
    assert got["status"] == simulee.ETIMEOUT
    stalled.close()
    assert diff(gpu_check(tr), oracle.check(tr)) == []
