"""Pins for the CPU oracle: what the paper and the mathematics fix, independently of the oracle.

* exhaustive all-pairs checks on tiny random traces (tests/bruteforce.py)
* the paper's worked examples (tests/golden/)
* hand-built cases with closed-form answers (tests/cases.py)
* generator families whose answers are known by construction
* metamorphic relations (record order, unit relabelling, sole-accessor reads)
"""
import numpy as np
import pytest

import oracle
import tracegen
from bruteforce import as_tuples, brute
import cases
import golden_io


@pytest.mark.parametrize("chunk", range(6))
def test_oracle_equals_all_pairs_on_tiny_traces(chunk):
    for seed in range(chunk * 100, chunk * 100 + 100):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 7 == 3))
        assert as_tuples(oracle.check(tr)) == brute(tr), f"seed {seed}"


def test_oracle_equals_all_pairs_hypothesis():
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(seed=st.integers(0, 2**31), n=st.integers(0, 60), nb=st.integers(1, 3), bt=st.integers(1, 6),
               me=st.integers(1, 4), units=st.integers(1, 5), pg=st.floats(0, 1), pa=st.floats(0, 0.5),
               unsorted=st.booleans())
    def prop(seed, n, nb, bt, me, units, pg, pa, unsorted):
        tr = tracegen.random_tiny(seed, n, nb, bt, me, units, p_global=pg, p_atomic=pa, unsorted=unsorted)
        assert as_tuples(oracle.check(tr)) == brute(tr)

    prop()


def test_dense_tiny_traces_have_every_kind_of_result():
    """The random family exercises all outputs (otherwise the all-pairs check proves little)."""
    kinds = np.zeros(6, dtype=int)
    for seed in range(300):
        o = oracle.check(tracegen.random_tiny(seed))
        r = o["races"]
        kinds += [len(r) > 0, (r["scope"] == 1).any(), (r["cls"] == 0).any(), len(o["divergence"]) > 0,
                  len(o["redundant"]) > 0, len(o["grid_redundant"]) > 0]
    assert (kinds > 20).all(), kinds


# ---- validation -------------------------------------------------------------------

@pytest.mark.parametrize("what,idx", cases.BAD_RECORDS)
def test_validation_reports_first_bad_record(what, idx):
    tr, want = cases.bad_record(what, idx)
    o = oracle.check(tr)
    assert (o["status"], o["bad_kind"], o["bad_index"]) == want
    assert as_tuples(o) == brute(tr)


def test_validation_counts_before_records():
    tr, want = cases.bad_count()
    o = oracle.check(tr)
    assert (o["status"], o["bad_kind"], o["bad_index"]) == want
    assert as_tuples(o) == brute(tr)


def test_unsorted_flag_accepts_any_order():
    tr = cases._valid_base()
    tr.events[:, 1] = tr.events[::-1, 1].copy()
    assert oracle.check(tr)["status"] == 2
    tr.flags = tracegen.UNSORTED
    assert oracle.check(tr)["status"] == 0


def test_empty_trace():
    b = tracegen.Builder(3, 5, 4, 4)
    b.set_counts(2)
    o = oracle.check(b.trace())
    assert o["status"] == 0 and len(o["races"]) == 0 and len(o["divergence"]) == 0
    # no accesses at all: every barrier is redundant (nothing can be reordered)
    assert [tuple(x) for x in o["redundant"]] == [(b_, k) for b_ in range(3) for k in range(2)]
    assert list(o["grid_redundant"]) == [0, 1]


# ---- the paper's worked examples ----------------------------------------------------

def test_golden_memory_unit_example():
    for tr, exp in golden_io.load("fig8_memory_unit.txt"):
        o = oracle.check(tr)
        assert o["status"] == 0
        assert golden_io.race_tuples(o) == exp["races"]
        assert [tuple(int(v) for v in x) for x in o["redundant"]] == exp["redundant"]
        assert len(o["divergence"]) == 0


def test_golden_kaldi_copy_from_mat():
    (tr, exp), = golden_io.load("kaldi_copy_from_mat.txt")
    o = oracle.check(tr)
    assert golden_io.race_tuples(o) == exp["races"]
    # the pair the text names: threads (1,0,0) and (0,1,0)
    assert (1, 3) in {(int(x["gtid_first"]), int(x["gtid_second"])) for x in o["races"]}


# ---- closed forms ----------------------------------------------------------------------

@pytest.mark.parametrize("name", sorted(cases.ALL))
def test_closed_form_cases(name):
    tr, exp = cases.ALL[name]()
    o = oracle.check(tr)
    assert cases.check_expect(o, exp) == []


def test_barrier_family_known_by_construction():
    tr = tracegen.barrier(seed=11, n_blocks=120, block_threads=128, n_epochs=24, shared_units=1024,
                          diverge_p=0.06, redirect_p=2e-4)
    o = oracle.check(tr)
    div = tr.meta["divergent_blocks"]
    assert len(div) > 0
    assert [int(x["block"]) for x in o["divergence"]] == list(div)
    assert all(int(x["min_count"]) == 22 and int(x["max_count"]) == 23 for x in o["divergence"])
    mask = tr.meta["redundant_mask"]
    R = [k for k in range(23) if (mask >> k) & 1]
    ds = set(int(b) for b in div)
    for blk in range(tr.n_blocks):
        if blk in ds:
            continue
        got = [int(x["barrier"]) for x in o["redundant"] if x["block"] == blk]
        assert got == R, blk
    # no barrier outside R is redundant anywhere, so the grid list is R minus
    # whatever the divergent blocks' mislabelled accesses made necessary
    assert set(int(k) for k in o["grid_redundant"]) <= set(R)


def test_strided_single_block_shape():
    tr = tracegen.c1()
    assert tr.n_events == 32768 and tr.n_blocks == 1 and tr.block_threads == 256
    acts = (tr.events[:, 3] >> 28) & 3
    frac_w = float((acts == 1).mean())
    assert 0.22 < frac_w < 0.28
    o = oracle.check(tr)
    assert o["status"] == 0 and len(o["races"]) > 0


# ---- metamorphic relations -------------------------------------------------------------

def _result_key(o):
    return as_tuples(o)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_record_permutation_with_unsorted_flag(seed):
    tr = tracegen.pattern(seed, n_blocks=6, block_threads=64, n_epochs=10, shared_units=2048, global_units=1 << 15)
    base = oracle.check(tr)
    perm = np.random.default_rng(seed).permutation(tr.n_events)
    tr2 = tracegen.Trace(tr.events[perm].copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                         tr.shared_units, tr.global_units, tr.max_barriers, tracegen.UNSORTED)
    assert _result_key(oracle.check(tr2)) == _result_key(base)


def test_unit_relabelling_permutes_keys():
    tr = tracegen.pattern(5, n_blocks=4, block_threads=64, n_epochs=8, shared_units=2048, global_units=1 << 15)
    base = oracle.check(tr)
    rng = np.random.default_rng(0)
    ps = rng.permutation(tr.shared_units).astype(np.uint32)
    pg = rng.permutation(tr.global_units).astype(np.uint32)
    ev = tr.events.copy()
    glob = ((ev[:, 3] >> 30) & 1) == 1
    ev[~glob, 0] = ps[ev[~glob, 0]]
    ev[glob, 0] = pg[ev[glob, 0]]
    tr2 = tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                         tr.global_units, tr.max_barriers)
    o2 = oracle.check(tr2)

    def mapped(o, fs, fg):
        s = set()
        for x in o["races"]:
            u = int(x["unit"])
            u = fg[u] if x["space"] == 1 else fs[u]
            s.add((int(x["space"]), int(x["scope"]), int(x["cls"]), int(x["block"]), int(x["epoch"]), int(u),
                   int(x["vo_first"]), int(x["vo_second"]), int(x["gtid_first"]), int(x["gtid_second"])))
        return s

    ident_s, ident_g = np.arange(tr.shared_units), np.arange(tr.global_units)
    assert mapped(base, ps, pg) == mapped(o2, ident_s, ident_g)
    assert _result_key(o2)["redundant"] == _result_key(base)["redundant"]


def test_reads_by_sole_accessor_change_nothing():
    tr = tracegen.pattern(9, n_blocks=4, block_threads=64, n_epochs=8, shared_units=2048, global_units=1 << 15)
    base = oracle.check(tr)
    ev = tr.events
    sh = ((ev[:, 3] >> 30) & 1) == 0
    key = ev[sh, 2].astype(np.int64) * tr.shared_units + ev[sh, 0]
    tid = ev[sh, 3] & 0xFFFF
    # (block, unit) pairs touched by exactly one thread
    order = np.lexsort((tid, key))
    k_s, t_s = key[order], tid[order]
    uniq, first = np.unique(k_s, return_index=True)
    last = np.r_[first[1:], len(k_s)] - 1
    sole = uniq[t_s[first] == t_s[last]][:50]
    sole_tid = t_s[first][t_s[first] == t_s[last]][:50]
    assert len(sole) > 10
    extra = []
    vo = int(ev[:, 1].max()) + 1
    for j, (k, t) in enumerate(zip(sole, sole_tid)):
        blk, unit = divmod(int(k), tr.shared_units)
        ep = int(tr.barrier_counts[blk * tr.block_threads + int(t)])
        extra.append(tracegen.pack(unit, vo + j, blk, int(t), ep, tracegen.READ, tracegen.SHARED))
    tr2 = tracegen.Trace(np.concatenate([ev] + extra), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                         tr.shared_units, tr.global_units, tr.max_barriers)
    assert _result_key(oracle.check(tr2)) == _result_key(base)
