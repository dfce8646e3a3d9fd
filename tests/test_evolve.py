"""The evolutionary search of Algorithms 1 and 2 (host logic, CPU) and the model-kernel traces it
scores. The host scorer here is the reference model generator plus the oracle's fitness; the GPU tests
check that the device generator and the batched device fitness give the same traces and the same
search trajectory."""
import math

import numpy as np
import pytest

import oracle
import tracegen
from paper_1905_01833_gb300 import evolve, simulee

SMALL = {simulee.MODEL_COPY2D: ((1, 1, 1, 1), (3, 3, 8, 8)), simulee.MODEL_STENCIL: ((1, 1, 1, 1), (4, 1, 64, 1))}


class OracleScorer:
    """Host scorer: the reference model generator and the oracle's fitness."""

    def __call__(self, sols):
        return [oracle.fitness(tracegen.model_trace(*s.launch())) for s in sols]


def test_copy2d_closed_forms():
    # row stride = width: every address has one thread, F = 1 (the paper's "no conflict" maximum)
    tr = tracegen.model_trace(tracegen.MODEL_COPY2D, (2, 3), (4, 5), (8, 8))
    f = oracle.fitness(tr)
    assert (f["n_addresses"], f["n_pairs"]) == (2 * 120, 2 * 120)
    # stride 0: every row hits the same X range, 32 addresses per array, 1024 thread pairs each
    tr = tracegen.model_trace(tracegen.MODEL_COPY2D, (1, 1), (32, 32), (0, 0))
    f = oracle.fitness(tr)
    assert (f["n_addresses"], f["n_pairs"]) == (64, 2048)
    # kaldi's _copy_from_mat (Sec. 2): block (3, 2), stride 1: threads (1,0) and (0,1) both write dst[1]
    tr = tracegen.model_trace(tracegen.MODEL_COPY2D, (1, 1), (3, 2), (1, 1))
    ww = [r for r in oracle.check(tr)["races"] if r["cls"] == 0]
    assert [(int(r["gtid_first"]), int(r["gtid_second"])) for r in ww] == [(1, 3), (2, 4)]


def test_stencil_closed_forms():
    # unit stride, no shift: every thread keeps to its own shared unit; the barrier is redundant
    tr = tracegen.model_trace(tracegen.MODEL_STENCIL, (2, 1), (16, 1), (0, 1))
    f, c = oracle.fitness(tr), oracle.check(tr)
    assert f["n_addresses"] == f["n_pairs"] == 2 * 16 + 32
    assert len(c["races"]) == 0 and len(c["redundant"]) == 2
    # shift by one: thread t reads what thread t+1 wrote before the barrier: the barrier is needed
    tr = tracegen.model_trace(tracegen.MODEL_STENCIL, (1, 1), (16, 1), (1, 1))
    c = oracle.check(tr)
    assert len(c["races"]) == 0 and len(c["redundant"]) == 0
    # stride 0: all threads write shared unit 0 before the barrier: write-write race
    tr = tracegen.model_trace(tracegen.MODEL_STENCIL, (1, 1), (8, 1), (0, 0))
    assert [int(r["cls"]) for r in oracle.check(tr)["races"]] == [0]


def test_scores_and_rank_rule():
    fit = dict(n_addresses=3, n_pairs=12, shared_lo=0xFFFFFFFF, shared_hi=0, global_lo=5, global_hi=9)
    assert evolve.scores(fit) == (0.25, 4)
    assert evolve.scores(dict(fit, n_addresses=0, n_pairs=0))[0] == 1.0
    S = evolve.Solution
    a, b, c = S(0, (1, 1, 1, 1), (0, 0), 1.0, 9), S(0, (1, 1, 1, 1), (0, 0), 1.0, 3), S(0, (1, 1, 1, 1), (0, 0), 0.5, 99)
    assert evolve.rank([a, b, c])[0] is c              # F first
    assert evolve.rank([a, b]) == [b, a]               # all F = 1: R decides


def test_mutation_follows_algorithm_2():
    ev = evolve.Evolution(simulee.MODEL_COPY2D, OracleScorer(), seed=3, limits=SMALL[simulee.MODEL_COPY2D])
    p = evolve.Solution(simulee.MODEL_COPY2D, (2, 2, 4, 4), (10.0, 20.0))
    rng = np.random.default_rng(3)
    n, dn = rng.standard_normal(2), rng.integers(-1, 2, size=4)
    c_, dc = rng.standard_cauchy(2), rng.integers(-1, 2, size=4)
    kids = ev.mutate(p)
    assert kids[0].args == tuple(float(v) for v in np.asarray(p.args) + n)
    assert kids[1].args == tuple(float(v) for v in np.asarray(p.args) + c_)
    assert kids[0].dims == ev._clamp_dims(np.asarray(p.dims) + dn)
    assert all(abs(a - b) <= 1 for a, b in zip(kids[1].dims, p.dims))


@pytest.mark.parametrize("model", [simulee.MODEL_COPY2D, simulee.MODEL_STENCIL])
def test_search_is_reproducible_and_never_worse(model):
    runs = [evolve.Evolution(model, OracleScorer(), population=12, generations=3, seed=11,
                             limits=SMALL[model]).run() for _ in range(2)]
    a, b = runs
    assert [(s.dims, s.args, s.F, s.R) for s in a["population"]] == [(s.dims, s.args, s.F, s.R) for s in b["population"]]
    fs = [f for f, _ in a["history"]]
    assert all(y <= x for x, y in zip(fs, fs[1:]))     # survivors include the parents
    assert a["population"] == evolve.rank(a["population"])
    assert all(not math.isnan(s.F) for s in a["population"])


def test_search_finds_an_acceptable_copy2d_launch():
    r = evolve.Evolution(simulee.MODEL_COPY2D, OracleScorer(), population=20, generations=6, seed=5,
                         limits=SMALL[simulee.MODEL_COPY2D], init_arg_range=8.0).run()
    assert r["accepted"] and r["best"].F < 0.3
