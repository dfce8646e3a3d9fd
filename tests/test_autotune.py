"""Autotuner: shape buckets, knobs and the cache round trip (CPU); tuned single and batched checks equal the
oracle (GPU)."""
import json

import pytest

import tracegen


def test_buckets_and_knobs():
    from paper_1905_01833_gb300 import autotune

    class T:
        n_events, n_blocks, max_barriers, block_threads = 61_000_000, 1024, 31, 256
    assert autotune.bucket(T) == "n26-b10-e5"

    class W(T):
        flags = tracegen.WARP_AWARE
    assert autotune.bucket(W) == "n26-b10-e5-f2"   # warp-aware traces take the sort: a bucket of their own
    assert autotune.batch_bucket([T, T]) == "batch-t1-n27-s4"
    # every knob's first value is the library's default (0 in simulee_options selects it)
    assert autotune.DEFAULTS == {"path": 0, "hash_shape": 0, "hash_cap_eighths": 7, "hash_pool_div": 3,
                                 "hot_unit_marks": 0, "hash_groups": 0, "sort_items": 16, "radix_bits": 8, "ingest_ctas_per_sm": 2,
                                 "sort_ctas_per_sm": 3, "reduce_ctas_per_sm": 3}
    for k in ("sort_items", "radix_bits", "hash_cap_eighths", "hash_pool_div", "hot_unit_marks", "hash_groups"):
        assert len(autotune.KNOBS[k]) >= 2


def test_descent_keeps_the_fastest(tmp_path):
    from paper_1905_01833_gb300 import autotune
    tuner = autotune.Autotuner.__new__(autotune.Autotuner)
    # a made-up cost: 11-bit digits and the smaller tile are faster, the sort path is slower
    cost = lambda o: 10.0 - (o["radix_bits"] == 11) - 0.5 * (o["sort_items"] == 8) + 5 * (o["path"] == 1)
    best, ms, log = tuner._descend(cost)
    assert best["radix_bits"] == 11 and best["sort_items"] == 8 and best["path"] == 0
    assert ms == 8.5 and min(m for _, m in log) == ms


@pytest.mark.gpu
def test_tuned_options_give_the_same_results(tmp_path):
    import oracle
    from paper_1905_01833_gb300 import autotune, simulee
    from gpu_util import diff
    tr = tracegen.pattern(5, n_blocks=24, block_threads=256, n_epochs=16, shared_units=12288, global_units=1 << 20)
    dt = simulee.to_device(tr)
    tuner = autotune.Autotuner(0, cache_path=str(tmp_path / "cache.json"))
    best = tuner.tune(dt, reps=1, sweeps=1)
    cache = json.load(open(tmp_path / "cache.json"))
    assert tuner.key(dt) in cache and all(k in cache[tuner.key(dt)] for k in autotune.KNOBS)
    assert autotune.Autotuner(0, cache_path=str(tmp_path / "cache.json")).best(dt) == best
    assert diff(tuner.checker(dt).check(dt), oracle.check(tr)) == []


@pytest.mark.gpu
def test_tuned_batch_equals_oracle(tmp_path):
    import oracle
    from paper_1905_01833_gb300 import autotune, simulee
    from gpu_util import diff
    sizes, bss, eps = tracegen.c3_sizes(seed=9, n_traces=40, median=2e4, sigma=0.9, lo=500, hi=3e5)
    trs = [tracegen.c3_trace(i, int(n), int(b), int(e), seed=9) for i, (n, b, e) in enumerate(zip(sizes, bss, eps))]
    dts = [simulee.to_device(t) for t in trs]
    tuner = autotune.Autotuner(0, cache_path=str(tmp_path / "cache.json"))
    best = tuner.tune_batch(dts, reps=1, sweeps=1)
    hit = json.load(open(tmp_path / "cache.json"))[tuner.batch_key(dts)]
    assert all(k in hit for k in autotune.KNOBS) and hit["evaluated"] >= 8   # the hash knobs are skipped once the sort path wins
    got = simulee.Checker(0, **best).check_batch(dts, compact=True)
    for i, t in enumerate(trs):
        assert diff(got[i], oracle.check(t)) == [], f"trace {i}"


@pytest.mark.gpu
@pytest.mark.parametrize("opts", [dict(radix_bits=6), dict(radix_bits=11), dict(sort_items=8),
                                  dict(radix_bits=11, sort_items=8, path=1), dict(radix_bits=6, path=1),
                                  dict(hash_cap_eighths=4, hash_pool_div=64), dict(hot_unit_marks=2)])
def test_every_knob_value_equals_oracle(opts):
    """Each sort width and tile, and the tightest hash cutover, on traces that send records through every stream
    (unsorted and warp-aware traces, a spilling grid trace) in one batch."""
    import oracle
    from paper_1905_01833_gb300 import simulee
    from gpu_util import diff
    trs = [tracegen.pattern(3, n_blocks=40, block_threads=256, n_epochs=12, shared_units=12288, global_units=1 << 20),
           tracegen.c1(), tracegen.random_tiny(4, unsorted=True, n_events=600),
           tracegen.with_statements(tracegen.random_grouped(8, n_events=500))]
    got = simulee.Checker(0, **opts).check_batch([simulee.to_device(t) for t in trs])
    for i, t in enumerate(trs):
        assert diff(got[i], oracle.check(t)) == [], f"{opts} trace {i}"
