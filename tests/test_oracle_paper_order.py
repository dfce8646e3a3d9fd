"""Pins of the oracle's paper visit-order variant (flag PAPER_ORDER).

Algorithm 3 keeps a visit-order counter per memory address, restarted at 0 for
every block (global addresses included), and a barrier bumps an address's
counter only when the address was visited since its last bump. Algorithm 5
groups a unit's tuples by visit order. Compared with grouping by epoch, this
changes two things, each pinned here by a hand-built trace whose answer
follows by inspection: a barrier is judged against a unit's next non-empty
epoch (empty epochs are skipped), and global accesses of different blocks meet
only at equal visit orders. Everything is also checked against the all-pairs
brute force (which replays the counters epoch by epoch), and planted mistakes
in the oracle source must each fail a pin.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import tracegen
from bruteforce import as_tuples, brute

R, W, A = tracegen.READ, tracegen.WRITE, tracegen.ATOMIC
SH, GL = tracegen.SHARED, tracegen.GLOBAL


def _trace(rows, n_blocks=1, bt=8, counts=2, paper=True):
    """rows: (block, tid, epoch, unit, action, space) in schedule order."""
    b = tracegen.Builder(n_blocks, bt, 64, 64)
    for blk, tid, ep, unit, act, sp in rows:
        b.access(blk, tid, ep, unit, act, sp)
    tr = b.set_counts(counts).trace()
    if paper:
        tr.flags |= tracegen.PAPER_ORDER
    return tr


def _races(tr, lib=None):
    return [(int(r["space"]), int(r["scope"]), int(r["cls"]), int(r["block"]), int(r["epoch"]), int(r["unit"]),
             int(r["gtid_first"]), int(r["gtid_second"])) for r in oracle.check(tr, lib=lib)["races"]]


def _redundant(tr, lib=None):
    return [(int(r["block"]), int(r["barrier"])) for r in oracle.check(tr, lib=lib)["redundant"]]


NONE = 0xFFFFFFFF
# name: (rows, n_blocks, counts, races (paper), redundant (paper), races (epochs), redundant (epochs))
CASES = {
    # a write in epoch 0, a read by another thread in epoch 2, nothing in epoch 1: the unit's
    # counter goes 0 -> 1 at barrier 0 only, so barrier 0 separates the two (needed), barrier 1
    # bumps nothing (redundant); by epochs no pair is adjacent and both are redundant
    "gap_barrier": ([(0, 1, 0, 5, W, SH), (0, 2, 2, 5, R, SH)], 1, 2,
                    [], [(0, 1)], [], [(0, 0), (0, 1)]),
    # the same with two empty epochs between: still barrier 0
    "gap_of_two": ([(0, 1, 0, 5, W, SH), (0, 2, 3, 5, R, SH)], 1, 3,
                   [], [(0, 1), (0, 2)], [], [(0, 0), (0, 1), (0, 2)]),
    # reads only across the gap: nothing conflicts, every barrier redundant either way
    "gap_reads": ([(0, 1, 0, 5, R, SH), (0, 2, 2, 5, R, SH)], 1, 2,
                  [], [(0, 0), (0, 1)], [], [(0, 0), (0, 1)]),
    # block 1 first touches global unit 7 in epoch 3: its counter is 0 there, like block 0's in
    # epoch 0, so the write and the read meet (RW, visit order 0); by epochs they race as well
    "inter_same_order": ([(0, 0, 0, 7, W, GL), (1, 0, 3, 7, R, GL)], 2, 3,
                         [(1, 1, 1, NONE, 0, 7, 0, 8)], [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 2)],
                         [(1, 1, 1, NONE, NONE, 7, 0, 8)], [(0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (1, 2)]),
    # block 0 reads unit 7 (order 0) then writes it (order 1); block 1 only reads it (order 0):
    # no write shares an order with the other block's read, so no race; by epochs RW
    "inter_orders_differ": ([(0, 0, 0, 7, R, GL), (1, 0, 0, 7, R, GL), (0, 0, 1, 7, W, GL)], 2, 1,
                            [], [(0, 0), (1, 0)],
                            [(1, 1, 1, NONE, NONE, 7, 8, 0)], [(0, 0), (1, 0)]),
    # two orders that both race: one inter record per order, epoch field = the order
    "inter_two_orders": ([(0, 0, 0, 9, W, GL), (1, 1, 1, 9, R, GL), (0, 0, 2, 9, W, GL), (1, 1, 5, 9, R, GL)], 2, 5,
                         [(1, 1, 1, NONE, 0, 9, 0, 9), (1, 1, 1, NONE, 1, 9, 0, 9)],
                         [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 0), (1, 1), (1, 2), (1, 3), (1, 4)],
                         [(1, 1, 1, NONE, NONE, 9, 0, 9)],
                         [(0, 0), (0, 1), (0, 2), (0, 3), (0, 4), (1, 0), (1, 1), (1, 2), (1, 3), (1, 4)]),
    # inside a block orders and epochs group alike: an intra-block race is the same record
    "intra_unchanged": ([(0, 1, 1, 3, W, SH), (0, 2, 1, 3, R, SH)], 1, 2,
                        [(0, 0, 1, 0, 1, 3, 1, 2)], [(0, 0), (0, 1)],
                        [(0, 0, 1, 0, 1, 3, 1, 2)], [(0, 0), (0, 1)]),
    # two reads of one epoch count once: block 0's write in epoch 1 has order 1 (not 2) and meets
    # block 1's read of order 1
    "inter_repeat_in_epoch": ([(0, 0, 0, 7, R, GL), (0, 1, 0, 7, R, GL), (1, 2, 0, 7, R, GL), (0, 0, 1, 7, W, GL),
                               (1, 2, 1, 7, R, GL)], 2, 1,
                              [(1, 1, 1, NONE, 1, 7, 0, 10)], [(1, 0)],
                              [(1, 1, 1, NONE, NONE, 7, 10, 0)], [(1, 0)]),
    # counters are per unit: block 0's earlier access to unit 3 leaves unit 7's write at order 0
    "inter_rank_per_unit": ([(0, 0, 0, 3, R, GL), (1, 1, 0, 7, R, GL), (0, 0, 1, 7, W, GL)], 2, 1,
                            [(1, 1, 1, NONE, 0, 7, 9, 0)], [(0, 0), (1, 0)],
                            [(1, 1, 1, NONE, NONE, 7, 9, 0)], [(0, 0), (1, 0)]),
    # and per space: shared unit 7 of block 0 is another address than global unit 7
    "inter_rank_per_space": ([(0, 0, 0, 7, R, SH), (1, 1, 0, 7, R, GL), (0, 0, 1, 7, W, GL)], 2, 1,
                             [(1, 1, 1, NONE, 0, 7, 9, 0)], [(0, 0), (1, 0)],
                             [(1, 1, 1, NONE, NONE, 7, 9, 0)], [(0, 0), (1, 0)]),
    # another unit in between does not close the gap: unit 5 (epochs 0, 2) keeps barrier 0 needed,
    # unit 6 (epoch 1 only) adds nothing
    "gap_other_unit": ([(0, 1, 0, 5, W, SH), (0, 3, 1, 6, W, SH), (0, 2, 2, 5, R, SH)], 1, 2,
                       [], [(0, 1)], [], [(0, 0), (0, 1)]),
}


def _pins_fail(lib):
    for name, (rows, nb, counts, rp, dp, re_, de) in CASES.items():
        for paper, rw, dw in ((True, rp, dp), (False, re_, de)):
            tr = _trace(rows, n_blocks=nb, counts=counts, paper=paper)
            if _races(tr, lib) != rw:
                return f"{name} races (paper={paper})"
            if _redundant(tr, lib) != dw:
                return f"{name} redundant (paper={paper})"
    return None


def test_paper_order_pins():
    assert _pins_fail(None) is None


@pytest.mark.parametrize("name", sorted(CASES))
def test_case(name):
    rows, nb, counts, rp, dp, re_, de = CASES[name]
    tr = _trace(rows, n_blocks=nb, counts=counts)
    assert _races(tr) == rp
    assert _redundant(tr) == dp
    assert as_tuples(oracle.check(tr)) == brute(tr)


@pytest.mark.parametrize("chunk", range(4))
def test_oracle_equals_all_pairs(chunk):
    for seed in range(chunk * 50, chunk * 50 + 50):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 7 == 3))
        tr.flags |= tracegen.PAPER_ORDER
        assert as_tuples(oracle.check(tr)) == brute(tr), seed


def test_oracle_equals_all_pairs_hypothesis():
    """Random shapes, sizes, spaces and action mixes (more epochs than units, so units skip epochs)."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2**31), n=st.integers(0, 60), nb=st.integers(1, 3), bt=st.integers(1, 6),
               me=st.integers(1, 6), units=st.integers(1, 5), pg=st.floats(0, 1), pa=st.floats(0, 0.5),
               unsorted=st.booleans())
    def prop(seed, n, nb, bt, me, units, pg, pa, unsorted):
        tr = tracegen.random_tiny(seed, n, nb, bt, me, units, p_global=pg, p_atomic=pa, unsorted=unsorted)
        tr.flags |= tracegen.PAPER_ORDER
        assert as_tuples(oracle.check(tr)) == brute(tr)

    prop()


def test_against_epoch_grouping():
    """Intra-block races are the same records; the variant only adds needed barriers (a unit's
    next non-empty epoch after k is k + 1 whenever epoch k + 1 touches it)."""
    for seed in range(60):
        tr = tracegen.random_tiny(seed, max_epochs=6)
        tp = tracegen.Trace(tr.events, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                            tr.global_units, tr.max_barriers, tr.flags | tracegen.PAPER_ORDER)
        a, b = oracle.check(tr), oracle.check(tp)
        ia, ib = a["races"][a["races"]["scope"] == 0], b["races"][b["races"]["scope"] == 0]
        assert ia.tobytes() == ib.tobytes(), seed
        red = lambda o: {(int(r["block"]), int(r["barrier"])) for r in o["redundant"]}
        assert red(b) <= red(a), seed
        assert a["divergence"].tobytes() == b["divergence"].tobytes()


def test_single_block_without_gaps_equals_epoch_grouping():
    """One block whose every unit is touched in every epoch from its first to its last: the
    counters equal the epochs minus a constant per unit, so both readings give the same output."""
    rng = np.random.default_rng(3)
    for seed in range(20):
        b = tracegen.Builder(1, 8, 16, 16)
        for e in range(4):
            for u in range(6):
                for _ in range(int(rng.integers(1, 3))):
                    b.access(0, int(rng.integers(0, 8)), e, u, int(rng.choice([R, W, A])),
                             SH if u % 2 else GL)
        tr = b.set_counts(3).trace()
        tp = tracegen.Trace(tr.events, tr.barrier_counts, 1, 8, 16, 16, tr.max_barriers, tracegen.PAPER_ORDER)
        a, p = oracle.check(tr), oracle.check(tp)
        for k in ("races", "redundant", "grid_redundant", "divergence"):
            assert a[k].tobytes() == p[k].tobytes(), (seed, k)


MUTANTS = {
    "adjacency_by_epoch": ("            (paper || (k[e].k1 & 0xFFFFFFFFu) == (k[s].k1 & 0xFFFFFFFFu) + 1)) {",
                           "            (0 || (k[e].k1 & 0xFFFFFFFFu) == (k[s].k1 & 0xFFFFFFFFu) + 1)) {"),
    "inter_by_unit": ("        k[m].k0 = paper ? r[i].rank : r[i].unit; k[m].k1 = paper ? r[i].unit : 0;",
                      "        k[m].k0 = r[i].unit; k[m].k1 = 0;"),
    "rank_counts_records": ("        else if (k[i].k1 != k[i - 1].k1) rank++;", "        else rank++;"),
    "rank_not_reset_per_unit": ("        if (i == 0 || k[i].k0 != k[i - 1].k0 || (k[i].k1 >> 32) != (k[i - 1].k1 >> 32)) rank = 0;",
                                "        if (i == 0 || k[i].k0 != k[i - 1].k0) rank = 0;"),
    "inter_epoch_field": ("        x.epoch = inter ? (paper ? q->rank : 0xFFFFFFFFu) : q->epoch;",
                          "        x.epoch = inter ? 0xFFFFFFFFu : q->epoch;"),
    "rank_per_space_ignored": ("        k[i].k0 = ((uint64_t)r[i].space << 32) | r[i].block;\n        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;\n        k[i].k2 = 0;",
                               "        k[i].k0 = r[i].block;\n        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;\n        k[i].k2 = 0;"),
}


@pytest.fixture(scope="module")
def src():
    oracle.build()
    return open(oracle._SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_paper_order_mutant_is_caught(name, src, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libpaper_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load(so)
    caught = _pins_fail(lib) is not None
    if not caught:   # the all-pairs comparison on tiny traces, with this build
        for seed in range(120):
            tr = tracegen.random_tiny(seed)
            tr.flags |= tracegen.PAPER_ORDER
            if as_tuples(oracle.check(tr, lib=lib)) != brute(tr):
                caught = True
                break
    assert caught, f"mutant {name} passed every pin"
    os.remove(so)
