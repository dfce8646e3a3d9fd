"""Continuous-batching server: every job's result equals the result of checking
its trace alone, whatever it was batched and overlapped with."""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import checker, diff

pytestmark = pytest.mark.gpu


def _pool():
    trs = [tracegen.pattern(s, n_blocks=2 + s % 5, block_threads=(64, 128, 256)[s % 3], n_epochs=6 + s % 9,
                            shared_units=12288, global_units=1 << 18) for s in range(8)]
    trs += [tracegen.random_tiny(s, n_events=500) for s in range(4)]
    trs += [tracegen.barrier(seed=4, n_blocks=8, block_threads=128, n_epochs=10, shared_units=1024, diverge_p=0.3),
            tracegen.c1(), tracegen.random_tiny(77, unsorted=True, n_events=300)]
    return trs


def _serve(trs, arrivals, **kw):
    from paper_1905_01833_gb300 import serve, simulee
    dts = [simulee.to_device(t) for t in trs]
    jobs = [serve.Job(i, dts[i % len(dts)], float(a)) for i, a in enumerate(arrivals)]
    srv = serve.Server(0, **kw)
    stats = srv.run(jobs)
    return jobs, stats


def test_served_results_equal_alone_results():
    from paper_1905_01833_gb300 import serve, simulee
    trs = _pool()
    alone = [checker().check(simulee.to_device(t)) for t in trs]
    arrivals = serve.poisson_arrivals(rate=5000.0, n=60, seed=1)
    jobs, stats = _serve(trs, arrivals)
    assert stats["max_batch"] > 1, stats          # jobs were batched
    for j in jobs:
        k = j.jid % len(trs)
        assert diff(j.result, alone[k]) == [], f"job {j.jid}"
        assert diff(j.result, oracle.check(trs[k])) == [], f"job {j.jid}"
    assert all(j.done >= j.arrival for j in jobs)


def test_batches_overlap_on_the_device():
    """A large job first (a few milliseconds of GPU work), then small jobs arriving while it runs: the
    later jobs are launched as further batches before the first one finishes, and every result still
    equals the result of checking the trace alone."""
    from paper_1905_01833_gb300 import serve, simulee
    big = tracegen.pattern(31, n_blocks=384, block_threads=256, n_epochs=32, shared_units=12288, global_units=1 << 22)
    trs = [big] + _pool()[:6]
    alone = [checker().check(simulee.to_device(t)) for t in trs]
    arrivals = [0.0] + [2e-4 * (k + 1) for k in range(12)]
    dts = [simulee.to_device(t) for t in trs]
    jobs = [serve.Job(0, dts[0], 0.0)] + [serve.Job(k + 1, dts[1 + k % 6], a) for k, a in enumerate(arrivals[1:])]
    stats = serve.Server(0, max_inflight=3).run(jobs)
    assert stats["max_inflight"] >= 2, stats      # batches overlapped on the device
    for j in jobs:
        k = 0 if j.jid == 0 else 1 + (j.jid - 1) % 6
        assert diff(j.result, alone[k]) == [], f"job {j.jid}"


def test_tight_budget_still_serves_everything():
    from paper_1905_01833_gb300 import serve
    trs = _pool()[:6]
    arrivals = serve.poisson_arrivals(rate=2000.0, n=20, seed=2)
    jobs, stats = _serve(trs, arrivals, hbm_budget=200 << 20)
    assert stats["max_reserved_bytes"] <= 200 << 20
    for j in jobs:
        assert diff(j.result, oracle.check(trs[j.jid % len(trs)])) == []


def test_serial_mode_matches():
    from paper_1905_01833_gb300 import serve
    trs = _pool()[:5]
    arrivals = serve.poisson_arrivals(rate=3000.0, n=15, seed=3)
    jobs, stats = _serve(trs, arrivals, serial=True)
    assert stats["max_batch"] == 1 and stats["max_inflight"] == 1
    for j in jobs:
        assert diff(j.result, oracle.check(trs[j.jid % len(trs)])) == []
