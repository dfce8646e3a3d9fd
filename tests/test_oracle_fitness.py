"""Pins of the oracle's fitness (Eq. 1 of the paper): F = sum g(i) / sum f(i).

f(i) is the number of distinct threads that access memory address i and g(i)
is 1 when address i is accessed; an address is a global unit or a shared unit
of one block. The pins do not retype the oracle's counting (a sort of
(address, thread) tuples): they count the same sums another way (per thread:
sum f = sum over threads of the number of distinct addresses the thread
touched), check closed forms of hand-built traces (private units give F = 1,
the paper's "no memory-access conflict" maximum), and plant mistakes in
copies of the oracle source, each of which must fail a pin.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import tracegen
import cases

EMPTY = 0xFFFFFFFF


def per_thread_count(tr):
    """sum g and sum f by a different route: per-thread address sets, then their union."""
    ev = tr.events.reshape(-1, 4)
    by_thread = {}
    ranges = {0: [EMPTY, 0], 1: [EMPTY, 0]}
    for unit, _vo, block, w3 in ev.tolist():
        space, tid = (w3 >> 30) & 1, w3 & 0xFFFF
        addr = (space, 0 if space else block, unit)
        by_thread.setdefault(block * tr.block_threads + tid, set()).add(addr)
        lo_hi = ranges[space]
        lo_hi[0], lo_hi[1] = min(lo_hi[0], unit), max(lo_hi[1], unit)
    n_pairs = sum(len(a) for a in by_thread.values())
    n_addr = len(set().union(*by_thread.values())) if by_thread else 0
    return n_addr, n_pairs, ranges


def _fields(o):
    return (o["n_addresses"], o["n_pairs"], {0: [o["shared_lo"], o["shared_hi"]], 1: [o["global_lo"], o["global_hi"]]})


def _pins_fail(lib) -> str | None:
    for seed in range(200):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 5 == 1))
        o = oracle.fitness(tr, lib=lib)
        if o["status"] != 0 or _fields(o) != per_thread_count(tr):
            return f"per-thread count seed {seed}"
    for name, mk in CLOSED.items():
        tr, want = mk()
        o = oracle.fitness(tr, lib=lib)
        if (o["n_addresses"], o["n_pairs"]) != want:
            return f"closed form {name}"
    for what, idx in cases.BAD_RECORDS:
        tr, want = cases.bad_record(what, idx)
        o = oracle.fitness(tr, lib=lib)
        if (o["status"], o["bad_kind"], o["bad_index"]) != want:
            return f"validation {what}"
    return None


def _private_units():
    # every thread of 3 blocks x 8 threads writes its own global unit in 3 epochs: F = 1
    b = tracegen.Builder(3, 8, 16, 64)
    for e in range(3):
        for blk in range(3):
            for t in range(8):
                b.access(blk, t, e, blk * 8 + t, tracegen.WRITE, tracegen.GLOBAL)
    return b.set_counts(2).trace(), (24, 24)


def _shared_broadcast():
    # every thread of each of 4 blocks reads shared unit 5: one address per block, 4 * 16 pairs
    b = tracegen.Builder(4, 16, 8)
    for blk in range(4):
        for t in range(16):
            b.access(blk, t, 0, 5, tracegen.READ)
    return b.set_counts(0).trace(), (4, 64)


def _global_broadcast():
    # every thread of 4 blocks reads global unit 5 twice: one address, 64 pairs
    b = tracegen.Builder(4, 16, 8, 8)
    for rep in range(2):
        for blk in range(4):
            for t in range(16):
                b.access(blk, t, rep, 5, tracegen.READ, tracegen.GLOBAL)
    return b.set_counts(1).trace(), (1, 64)


def _same_unit_both_spaces():
    # unit 3 in shared memory of blocks 0 and 1 and unit 3 in global memory are three addresses;
    # thread (1, 2) touches all three of them
    b = tracegen.Builder(2, 4, 8, 8)
    b.access(0, 1, 0, 3, tracegen.WRITE).access(1, 2, 0, 3, tracegen.WRITE)
    b.access(1, 2, 0, 3, tracegen.READ, tracegen.GLOBAL).access(0, 1, 0, 3, tracegen.ATOMIC, tracegen.GLOBAL)
    b.access(1, 2, 0, 3, tracegen.READ)
    return b.set_counts(0).trace(), (3, 4)


CLOSED = {"private_units": _private_units, "shared_broadcast": _shared_broadcast,
          "global_broadcast": _global_broadcast, "same_unit_both_spaces": _same_unit_both_spaces}


def test_oracle_fitness_passes_pins():
    assert _pins_fail(None) is None


@pytest.mark.parametrize("name", sorted(CLOSED))
def test_closed_forms(name):
    tr, (na, npairs) = CLOSED[name]()
    o = oracle.fitness(tr)
    assert (o["n_addresses"], o["n_pairs"]) == (na, npairs)
    assert o["n_addresses"] <= o["n_pairs"]


def test_private_units_give_the_maximum_fitness():
    tr, _ = _private_units()
    o = oracle.fitness(tr)
    assert o["n_addresses"] / o["n_pairs"] == 1.0


def test_validation_matches_the_check():
    for what, idx in cases.BAD_RECORDS:
        tr, _ = cases.bad_record(what, idx)
        f, c = oracle.fitness(tr), oracle.check(tr)
        assert (f["status"], f["bad_kind"], f["bad_index"]) == (c["status"], c["bad_kind"], c["bad_index"])
    tr, _ = cases.bad_count()
    f, c = oracle.fitness(tr), oracle.check(tr)
    assert (f["status"], f["bad_kind"], f["bad_index"]) == (c["status"], c["bad_kind"], c["bad_index"])


def test_empty_trace():
    tr = tracegen.Builder(2, 4, 8, 8).set_counts(0).trace()
    o = oracle.fitness(tr)
    assert (o["status"], o["n_addresses"], o["n_pairs"]) == (0, 0, 0)
    assert (o["shared_lo"], o["shared_hi"], o["global_lo"], o["global_hi"]) == (EMPTY, 0, EMPTY, 0)


MUTANTS = {
    "shared_not_per_block": ("        t[i].block = space ? 0u : block;\n", "        t[i].block = 0u;\n"),
    "thread_is_local_tid": ("        t[i].gtid = block * bt + tid;\n", "        t[i].gtid = tid;\n"),
    "counts_records": ("        *n_pairs += (uint64_t)new_pair;\n", "        *n_pairs += 1u;\n"),
    "space_ignored": ("        const int new_addr = i == 0 || t[i - 1].space != t[i].space || t[i - 1].block != t[i].block ||",
                      "        const int new_addr = i == 0 || t[i - 1].block != t[i].block ||"),
    "range_hi_min": ("        if (unit > *hi) *hi = unit;\n", "        if (unit < *hi) *hi = unit;\n"),
}


@pytest.fixture(scope="module")
def src():
    oracle.build()
    return open(oracle._SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_fitness_mutant_is_caught(name, src, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libfit_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load(so)
    assert _pins_fail(lib) is not None, f"mutant {name} passed every pin"
    os.remove(so)
