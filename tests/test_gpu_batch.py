"""Batched check on the GPU: every trace of a batch gets exactly the result it
gets alone (and the oracle's), in one batched call, whatever else is in the batch."""
import numpy as np
import pytest

import oracle
import tracegen
import cases
from gpu_util import checker, diff

pytestmark = pytest.mark.gpu


def _batch(trs, **kw):
    from paper_1905_01833_gb300 import simulee
    return checker().check_batch([simulee.to_device(t) for t in trs], **kw)


def test_batch_of_tiny_random_traces_equals_oracle():
    trs = [tracegen.random_tiny(s, unsorted=(s % 4 == 1)) for s in range(300)]
    for i, (got, tr) in enumerate(zip(_batch(trs), trs)):
        d = diff(got, oracle.check(tr))
        assert d == [], f"trace {i}: {d}"


def test_batch_mixed_shapes_equals_single_checks():
    from gpu_util import gpu_check
    sizes, bss, eps = tracegen.c3_sizes(seed=5, n_traces=24, median=4e3, sigma=0.87, lo=300, hi=3e4)
    trs = [tracegen.c3_trace(i, int(n), int(b), int(e), seed=5) for i, (n, b, e) in enumerate(zip(sizes, bss, eps))]
    trs.append(tracegen.c1())
    trs.append(tracegen.barrier(seed=2, n_blocks=6, block_threads=64, n_epochs=12, shared_units=512, diverge_p=0.3))
    got = _batch(trs)
    for i, tr in enumerate(trs):
        assert diff(got[i], gpu_check(tr)) == [], f"trace {i}"
        assert diff(got[i], oracle.check(tr)) == [], f"trace {i}"


def test_batch_isolates_bad_traces():
    good = [tracegen.random_tiny(s, n_events=80) for s in (11, 12, 13)]
    bad, want = cases.bad_record("epoch", 4)
    badc, wantc = cases.bad_count()
    trs = [good[0], bad, good[1], badc, good[2]]
    got = _batch(trs)
    assert (got[1]["status"], got[1]["bad_kind"], got[1]["bad_index"]) == want
    assert (got[3]["status"], got[3]["bad_kind"], got[3]["bad_index"]) == wantc
    for i in (0, 2, 4):
        assert diff(got[i], oracle.check(trs[i])) == []


def test_batch_truncates_per_trace():
    trs = [tracegen.c1(), tracegen.strided(seed=9)]
    want = [oracle.check(t) for t in trs]
    got = _batch(trs, races_caps=[50, 10**6])
    assert got[0]["status"] == 4 and got[0]["n_races"] == len(want[0]["races"])
    assert np.array_equal(got[0]["races"], want[0]["races"][:50])
    assert got[1]["status"] == 0 and np.array_equal(got[1]["races"], want[1]["races"])


def test_batch_with_empty_traces():
    b = tracegen.Builder(2, 4, 4, 4)
    b.set_counts(1)
    empty = b.trace()
    trs = [empty, tracegen.random_tiny(3), empty]
    for got, tr in zip(_batch(trs), trs):
        assert diff(got, oracle.check(tr)) == []
