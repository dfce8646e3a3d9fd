"""Device side of the evolutionary search: the model-kernel trace generator against the host
reference (byte for byte), the device scorer against the oracle scorer (the same search trajectory),
and the check of an accepted launch."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import checker, diff
from paper_1905_01833_gb300 import evolve, simulee
from test_evolve import SMALL, OracleScorer

pytestmark = pytest.mark.gpu


def _launches(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        model = int(rng.integers(0, 2))
        if model == simulee.MODEL_COPY2D:
            dims = ((int(rng.integers(1, 5)), int(rng.integers(1, 5))), (int(rng.integers(1, 33)), int(rng.integers(1, 17))))
        else:
            dims = ((int(rng.integers(1, 9)), 1), (int(rng.integers(1, 300)), 1))
        args = (int(rng.integers(-5, 5000)), int(rng.integers(-5, 70000)))
        out.append((model, dims[0], dims[1], args))
    return out


def test_device_traces_equal_host_traces():
    launches = _launches(1, 40) + [(0, (1, 1), (3, 2), (1, 1)), (1, (2, 1), (16, 1), (0, 1))]
    dts = checker().model_traces(launches)
    for (model, grid, block, args), dt in zip(launches, dts):
        tr = tracegen.model_trace(model, grid, block, args)
        assert np.array_equal(dt.events.cpu().numpy().view(np.uint32), tr.events), (model, grid, block, args)
        assert np.array_equal(dt.barrier_counts.cpu().numpy().view(np.uint32), tr.barrier_counts)
        assert (dt.n_blocks, dt.block_threads, dt.shared_units, dt.global_units, dt.max_barriers) == \
               (tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units, tr.max_barriers)


@pytest.mark.parametrize("model", [simulee.MODEL_COPY2D, simulee.MODEL_STENCIL])
def test_device_scorer_gives_the_oracle_trajectory(model):
    dev = evolve.Evolution(model, evolve.DeviceScorer(checker()), population=12, generations=3, seed=21,
                           limits=SMALL[model]).run()
    ref = evolve.Evolution(model, OracleScorer(), population=12, generations=3, seed=21, limits=SMALL[model]).run()
    assert [(s.dims, s.args, s.F, s.R) for s in dev["population"]] == \
           [(s.dims, s.args, s.F, s.R) for s in ref["population"]]
    assert dev["history"] == ref["history"]


def test_accepted_launch_is_checked():
    r = evolve.Evolution(simulee.MODEL_COPY2D, evolve.DeviceScorer(checker()), population=20, generations=6, seed=5,
                         limits=SMALL[simulee.MODEL_COPY2D], init_arg_range=8.0).run()
    assert r["accepted"]
    got = evolve.detect(checker(), r["best"])
    want = oracle.check(tracegen.model_trace(*r["best"].launch()))
    assert diff(got, want) == []
    assert len(got["races"]) > 0
