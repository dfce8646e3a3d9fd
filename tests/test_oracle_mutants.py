"""Planted mistakes: each mutant of the oracle source must fail at least one pin.

Every mutant is a plausible slip (a dropped term, a wrong index, a swapped
operand). The mutant is compiled from a copy of the oracle source on the CPU;
the real oracle is untouched. A mutant that passed every pin would show a gap
in the pins, so this file checks the pins themselves.
"""
import os
import subprocess

import pytest

import oracle
import tracegen
from bruteforce import as_tuples, brute
import cases
import golden_io

MUTANTS = {
    "both_atomic_rule_dropped": ("    if (p->act == ACT_A && q->act == ACT_A) return 0;\n", ""),
    "atomics_treated_as_reads": ("return act == ACT_W || act == ACT_A;", "return act == ACT_W;"),
    "same_owner_allowed": ("    if (id_p == id_q) return 0;\n", ""),
    "classes_swapped": ("? 0u : 1u;", "? 1u : 0u;"),
    "adjacency_off_by_one": ("(k[s].k1 & 0xFFFFFFFFu) + 1)", "(k[s].k1 & 0xFFFFFFFFu) + 2)"),
    "inter_owner_is_thread": ("uint32_t idq = inter ? rq->block : rq->gtid;", "uint32_t idq = rq->gtid;"),
    "latest_partner": ("for (uint64_t p = 0; p < q; p++) {", "for (uint64_t p = q; p-- > 0;) {"),
    "first_min_tid_last": ("if (c < mn) { mn = c; first = t; }", "if (c <= mn) { mn = c; first = t; }"),
    "epoch_check_strict": ("epoch > counts[(uint64_t)block * bt + tid]", "epoch >= counts[(uint64_t)block * bt + tid]"),
    "grid_past_last_barrier": ("for (uint32_t kk = 0; kk < gmax; kk++) {", "for (uint32_t kk = 0; kk <= gmax; kk++) {"),
    "pair_order_swapped": ("x.vo_first = p->vo; x.vo_second = q->vo;", "x.vo_first = q->vo; x.vo_second = p->vo;"),
    "inter_includes_shared": ("        if (r[i].space != 1) continue;\n", ""),
    "intra_ignores_epoch": ("k[i].k1 = ((uint64_t)r[i].epoch << 32) | r[i].unit;", "k[i].k1 = r[i].unit;"),
    "redundancy_ignores_space": ("k[i].k0 = ((uint64_t)r[i].space << 32) | r[i].block;\n        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;\n        k[i].k2 = r[i].vo;",
                                 "k[i].k0 = r[i].block;\n        k[i].k1 = ((uint64_t)r[i].unit << 32) | r[i].epoch;\n        k[i].k2 = r[i].vo;"),
    "vo_check_allows_equal": ("vo <= ev[4 * (i - 1) + 1]", "vo < ev[4 * (i - 1) + 1]"),
    "read_read_conflicts": ("    if (!modifies(p->act) && !modifies(q->act)) return 0;\n", ""),
}


def _pins_fail(lib) -> str | None:
    """Run the pins against a bound oracle build; return the first failing pin's name."""
    for seed in range(150):
        tr = tracegen.random_tiny(seed, unsorted=(seed % 7 == 3))
        if as_tuples(oracle.check(tr, lib=lib)) != brute(tr):
            return f"all-pairs seed {seed}"
    for name in ("fig8_memory_unit.txt", "kaldi_copy_from_mat.txt"):
        for tr, exp in golden_io.load(name):
            o = oracle.check(tr, lib=lib)
            if golden_io.race_tuples(o) != exp["races"]:
                return f"golden {name}"
            if exp["redundant"] is not None and [tuple(int(v) for v in x) for x in o["redundant"]] != exp["redundant"]:
                return f"golden {name} redundant"
    for what, idx in cases.BAD_RECORDS:
        tr, want = cases.bad_record(what, idx)
        o = oracle.check(tr, lib=lib)
        if (o["status"], o["bad_kind"], o["bad_index"]) != want:
            return f"validation {what}"
    tr, want = cases.bad_count()
    o = oracle.check(tr, lib=lib)
    if (o["status"], o["bad_kind"], o["bad_index"]) != want:
        return "validation counts"
    for name, mk in cases.ALL.items():
        tr, exp = mk()
        if cases.check_expect(oracle.check(tr, lib=lib), exp):
            return f"case {name}"
    return None


@pytest.fixture(scope="module")
def src():
    oracle.build()
    return open(oracle._SRC).read()


def test_real_oracle_passes_pins():
    assert _pins_fail(None) is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, src, tmp_path):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / f"libmutant_{name}.so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", so, str(path)])
    lib = oracle.load(so)
    assert _pins_fail(lib) is not None, f"mutant {name} passed every pin"
    os.remove(so)
