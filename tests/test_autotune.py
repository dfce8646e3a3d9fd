"""Autotuner: shape buckets and the cache round trip (CPU); tuned checking (GPU)."""
import json

import pytest

import tracegen


def test_bucket_and_candidates():
    from paper_1905_01833_gb300 import autotune

    class T:
        n_events, n_blocks, max_barriers = 61_000_000, 1024, 31
    assert autotune.bucket(T) == "n26-b10-e5"
    assert len(autotune.CANDIDATES) == 36
    assert all(set(c) == set(autotune.KNOBS) for c in autotune.CANDIDATES)


@pytest.mark.gpu
def test_tuned_options_give_the_same_results(tmp_path):
    import oracle
    from paper_1905_01833_gb300 import autotune, simulee
    from gpu_util import diff
    tr = tracegen.pattern(5, n_blocks=24, block_threads=256, n_epochs=16, shared_units=12288, global_units=1 << 20)
    dt = simulee.to_device(tr)
    tuner = autotune.Autotuner(0, cache_path=str(tmp_path / "cache.json"))
    best = tuner.tune(dt, reps=1, candidates=autotune.CANDIDATES[::5])
    cache = json.load(open(tmp_path / "cache.json"))
    assert tuner.key(dt) in cache
    assert autotune.Autotuner(0, cache_path=str(tmp_path / "cache.json")).best(dt) == best
    assert diff(tuner.checker(dt).check(dt), oracle.check(tr)) == []
