"""Pins of the oracle's warp-aware variant of Theorem 1 (traces with statement words).

Two accesses of threads in the same warp (same block, same tid / 32) race only
when both are plain writes of the same statement, or when either came after the
warp diverged; threads of different warps race as without the refinement.
Every pin is a hand-built trace whose answer follows from those three clauses
of Theorem 1 by inspection, including the paper's kaldi example (Sec. 2: the
two writes of one statement by threads of one warp); planted mistakes in the
oracle source must each fail a pin.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import tracegen

R, W, A = tracegen.READ, tracegen.WRITE, tracegen.ATOMIC
D = tracegen.DIVERGED


def _trace(rows, stmts, n_blocks=1, bt=64, counts=0):
    """rows: (block, tid, epoch, unit, action); stmts: statement word per row."""
    b = tracegen.Builder(n_blocks, bt, 64)
    for blk, tid, ep, unit, act in rows:
        b.access(blk, tid, ep, unit, act)
    tr = b.set_counts(counts).trace()
    tr.flags |= tracegen.WARP_AWARE
    tr.stmt = np.array(stmts, dtype=np.uint32)
    return tr


def _races(tr, lib=None):
    return [(int(r["cls"]), int(r["gtid_first"]), int(r["gtid_second"])) for r in oracle.check(tr, lib=lib)["races"]]


def _redundant(tr, lib=None):
    return [(int(r["block"]), int(r["barrier"])) for r in oracle.check(tr, lib=lib)["redundant"]]


CASES = {
    # threads 1 and 2 of warp 0: a write and a read of different statements, no divergence: no race
    "same_warp_read_write": (lambda: _trace([(0, 1, 0, 5, W), (0, 2, 0, 5, R)], [1, 2]), [], None),
    # the same with the write made after divergence: RW race
    "same_warp_diverged_write": (lambda: _trace([(0, 1, 0, 5, W), (0, 2, 0, 5, R)], [1 | D, 2]), [(1, 1, 2)], None),
    # the read diverged: RW race as well
    "same_warp_diverged_read": (lambda: _trace([(0, 1, 0, 5, W), (0, 2, 0, 5, R)], [1, 2 | D]), [(1, 1, 2)], None),
    # two writes of the same statement in one warp: WW race
    "same_warp_same_statement": (lambda: _trace([(0, 3, 0, 7, W), (0, 4, 0, 7, W)], [9, 9]), [(0, 3, 4)], None),
    # two writes of different statements in one warp: none
    "same_warp_two_statements": (lambda: _trace([(0, 3, 0, 7, W), (0, 4, 0, 7, W)], [9, 10]), [], None),
    # an atomic and a write of one statement id in one warp: not two writes, no race
    "same_warp_atomic_write": (lambda: _trace([(0, 3, 0, 7, A), (0, 4, 0, 7, W)], [9, 9]), [], None),
    # threads 1 and 33 are in different warps: RW race whatever the statements
    "different_warps": (lambda: _trace([(0, 1, 0, 5, W), (0, 33, 0, 5, R)], [1, 2]), [(1, 1, 33)], None),
    # same tid / 32 but different blocks (global memory): different warps, inter-block race
    "different_blocks": (lambda: (lambda t: t)(_global_pair()), None, None),
    # a barrier between a same-warp write and read of different statements: redundant under the refinement
    "barrier_same_warp": (lambda: _trace([(0, 1, 0, 5, W), (0, 2, 1, 5, R)], [1, 2], counts=1), [], [(0, 0)]),
    # the same barrier when the read is in another warp: needed
    "barrier_other_warp": (lambda: _trace([(0, 1, 0, 5, W), (0, 40, 1, 5, R)], [1, 2], counts=1), [], []),
}


def _global_pair():
    b = tracegen.Builder(2, 64, 64, 64)
    b.access(0, 1, 0, 5, W, tracegen.GLOBAL).access(1, 1, 0, 5, R, tracegen.GLOBAL)
    tr = b.set_counts(0).trace()
    tr.flags |= tracegen.WARP_AWARE
    tr.stmt = np.array([1, 2], dtype=np.uint32)
    return tr


def _kaldi():
    # Sec. 2, _copy_from_mat: block (3, 2), dst[y * 1 + x]; both writes to dst[1] come from one statement
    return tracegen.with_statements(tracegen.model_trace(tracegen.MODEL_COPY2D, (1, 1), (3, 2), (1, 1)),
                                    diverge_p=0.0)


def _pins_fail(lib):
    for name, (mk, races, red) in CASES.items():
        tr = mk()
        got = _races(tr, lib)
        if name == "different_blocks":
            if [(int(r["scope"]), int(r["cls"])) for r in oracle.check(tr, lib=lib)["races"]] != [(1, 1)]:
                return name
            continue
        if got != races:
            return name
        if red is not None and _redundant(tr, lib) != red:
            return name + " (redundant)"
    if [(c, a, b) for c, a, b in _races(_kaldi(), lib)] != [(0, 1, 3), (0, 2, 4)]:
        return "kaldi"
    # without statement words the refinement is off: the same-warp read/write pair races
    tr = CASES["same_warp_read_write"][0]()
    tr.flags &= ~tracegen.WARP_AWARE
    if _races(tr, lib) != [(1, 1, 2)]:
        return "flag off"
    return None


def test_warp_pins():
    assert _pins_fail(None) is None


@pytest.mark.parametrize("name", sorted(CASES))
def test_case(name):
    mk, races, red = CASES[name]
    tr = mk()
    if races is not None:
        assert _races(tr) == races
    if red is not None:
        assert _redundant(tr) == red


def test_full_divergence_equals_the_plain_check():
    """With every warp diverged the refinement never removes a pair: same result as without it."""
    for seed in range(40):
        tr = tracegen.random_tiny(seed)
        tw = tracegen.with_statements(tr, seed=seed, diverge_p=1.0)
        a, b = oracle.check(tr), oracle.check(tw)
        for k in ("races", "divergence", "redundant", "grid_redundant"):
            assert a[k].tobytes() == b[k].tobytes(), (seed, k)


def test_refinement_only_removes_pairs():
    """Warp-aware races are a subset (by group and class) of the plain ones, and needed barriers a subset."""
    for seed in range(40):
        tr = tracegen.random_tiny(seed, n_blocks=1, block_threads=70, units=6)
        tw = tracegen.with_statements(tr, seed=seed, diverge_p=0.3)
        key = lambda r: (int(r["space"]), int(r["scope"]), int(r["block"]), int(r["epoch"]), int(r["unit"]), int(r["cls"]))
        plain, aware = oracle.check(tr), oracle.check(tw)
        assert {key(r) for r in aware["races"]} <= {key(r) for r in plain["races"]}
        red = lambda o: {(int(r["block"]), int(r["barrier"])) for r in o["redundant"]}
        assert red(plain) <= red(aware)


MUTANTS = {
    "refinement_dropped": ("        if (!same_statement_writes && !diverged) return 0;\n", ""),
    "warp_across_blocks": ("    return p->block == q->block && (p->tid >> 5) == (q->tid >> 5);",
                           "    return (p->tid >> 5) == (q->tid >> 5);"),
    "divergence_ignored": ("        const int diverged = (p->stmt & STMT_DIVERGED) || (q->stmt & STMT_DIVERGED);",
                           "        const int diverged = 0;"),
    "any_same_statement": ("        const int same_statement_writes = p->act == ACT_W && q->act == ACT_W &&",
                           "        const int same_statement_writes = 1 &&"),
    "warp_of_64": ("    return p->block == q->block && (p->tid >> 5) == (q->tid >> 5);",
                   "    return p->block == q->block && (p->tid >> 6) == (q->tid >> 6);"),
}


@pytest.fixture(scope="module")
def src():
    oracle.build()
    return open(oracle._SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_warp_mutant_is_caught(name, src, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libwarp_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load(so)
    assert _pins_fail(lib) is not None, f"mutant {name} passed every pin"
    os.remove(so)


@pytest.mark.parametrize("chunk", range(3))
def test_oracle_equals_all_pairs_with_statement_words(chunk):
    """The all-pairs brute force with Theorem 1's warp clauses, written separately, on random traces
    with statement words (tiny blocks: every same-block pair shares a warp)."""
    from bruteforce import as_tuples, brute
    for seed in range(chunk * 80, chunk * 80 + 80):
        tr = tracegen.with_statements(tracegen.random_tiny(seed), seed=seed, diverge_p=0.3)
        assert as_tuples(oracle.check(tr)) == brute(tr), seed
