"""The five workloads at their full sizes, checked on the GPU and compared with the
CPU oracle on every output record (tolerance zero: this is integer work).

* grid (1024 blocks x 256 threads, 32 epochs, ~6.1e7 records) and barrier
  (1024 x 1024 threads, 64 epochs, 2^28 records): the whole trace through the
  oracle.
* batched (4096 traces, 6e8 records): every member's result from one batched
  call against the oracle on that member, plus a field-by-field comparison on
  a stratified sample (the largest members, every block size, the fewest and
  the most epochs).
* served (jobs drawn from the pool of log-uniform traces of 1e4..1e8 records):
  every served job's result against the oracle on its trace, with batches
  overlapping on the device.
The oracle runs in spawned processes (one per host core) while the GPU works.
"""
import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import diff, oracle_digests_async, result_digest

pytestmark = pytest.mark.gpu

BIG_RACES_CAP = 4_000_000   # race-list capacity for the whole-trace checks


def _local_checker():
    from paper_1905_01833_gb300 import simulee
    return simulee.Checker(0)


def _release(chk):
    """Give a large workspace back to the device before the next test."""
    import torch
    chk._ws = None
    chk.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_grid_and_barrier_workloads_whole_trace():
    from paper_1905_01833_gb300 import simulee
    pool, pending = oracle_digests_async([("c4", ("c4",), BIG_RACES_CAP), ("c2", ("c2",), BIG_RACES_CAP)], 2)
    try:
        chk = _local_checker()
        got = {k: chk.check(simulee.to_device(g()), races_cap=BIG_RACES_CAP)
               for k, g in (("c2", tracegen.c2), ("c4", tracegen.c4))}
        _release(chk)
        want = {k: (n, d) for k, n, d in pending.get(timeout=1800)}
    finally:
        pool.close()
        pool.join()
    for k in ("c2", "c4"):
        assert got[k]["status"] == 0, (k, got[k]["status"])
        assert result_digest(got[k], BIG_RACES_CAP) == want[k][1], f"{k}: GPU result differs from the oracle"
    # known by construction: the barrier family's divergent blocks (1%) and redundant barrier set
    c4 = tracegen.c4()
    assert np.array_equal(got["c4"]["divergence"]["block"], c4.meta["divergent_blocks"])


def test_batched_workload_every_member():
    import torch
    from paper_1905_01833_gb300 import simulee
    sigma = tracegen.c3_sigma()
    sizes, bss, eps = tracegen.c3_sizes(sigma=sigma)
    recipes = [("c3", i, int(n), int(b), int(e), tracegen.DEFAULT_SEED) for i, (n, b, e) in
               enumerate(zip(sizes, bss, eps))]
    caps = [min(2 * int(n) + 2, 1024 + int(n) // 8) for n in sizes]
    order = sorted(range(len(recipes)), key=lambda i: -sizes[i])
    pool, pending = oracle_digests_async([(i, recipes[i], caps[i]) for i in order])
    try:
        trs = [tracegen.c3_trace(*r[1:]) for r in recipes]
        assert sum(t.n_events for t in trs) == tracegen.C3_RECORDS
        n = sum(t.n_events for t in trs)
        ev = torch.empty((n, 4), dtype=torch.int32, device="cuda:0")
        cn = torch.empty(sum(t.barrier_counts.size for t in trs), dtype=torch.int32, device="cuda:0")
        dts, a, b = [], 0, 0
        for t in trs:
            k, c = t.n_events, t.barrier_counts.size
            ev[a:a + k].copy_(torch.from_numpy(t.events.view(np.int32)))
            cn[b:b + c].copy_(torch.from_numpy(t.barrier_counts.view(np.int32)))
            dts.append(simulee.DeviceTrace(ev[a:a + k], cn[b:b + c], t.n_blocks, t.block_threads, t.shared_units,
                                           t.global_units, t.max_barriers))
            a += k
            b += c
        chk = _local_checker()
        got = chk.check_batch(dts, races_caps=caps)
        _release(chk)
        del dts, ev, cn
        want = {i: d for i, _, d in pending.get(timeout=1800)}
    finally:
        pool.close()
        pool.join()
    bad = [i for i in range(len(trs)) if result_digest(got[i], caps[i]) != want[i]]
    assert not bad, f"{len(bad)} members differ from the oracle, first {bad[0]}: {diff(got[bad[0]], oracle.check(trs[bad[0]]))}"
    # stratified field-by-field comparison
    pick = set(order[:3])
    for bs in (64, 128, 256, 1024):
        pick.add(int(np.flatnonzero(bss == bs)[np.argmax(sizes[bss == bs])]))
    pick.add(int(np.argmin(eps)))
    pick.add(int(np.argmax(eps)))
    assert sizes[order[0]] >= 1_000_000 and eps.min() == 4 and eps.max() == 64
    for i in sorted(pick):
        d = diff(got[i], oracle.check(trs[i]))
        assert d == [], f"member {i}: {d}"


def test_served_workload_every_job():
    import torch
    from paper_1905_01833_gb300 import serve, simulee
    n_pool = 24
    sizes = tracegen.c5_pool_sizes(n_pool)
    cap = 1 << 20   # the server's per-job race list
    pool, pending = oracle_digests_async([(i, ("c5", i, float(sizes[i])), cap) for i in range(n_pool - 1, -1, -1)])
    try:
        trs = [tracegen.c5_member(i, sz) for i, sz in enumerate(sizes)]
        dts = [simulee.to_device(t) for t in trs]
        rng = np.random.default_rng(7)
        draws = np.exp(rng.uniform(np.log(1e4), np.log(1e8), size=300))
        pick = np.abs(np.log(draws)[:, None] - np.log(sizes)[None, :]).argmin(axis=1)
        arrivals = serve.poisson_arrivals(2000.0, 300, seed=11)
        jobs = [serve.Job(k, dts[int(pick[k])], float(arrivals[k])) for k in range(300)]
        srv = serve.Server(0, hbm_budget=120 << 30)
        stats = srv.run(jobs)
        del srv
        torch.cuda.empty_cache()
        want = {i: d for i, _, d in pending.get(timeout=1800)}
    finally:
        pool.close()
        pool.join()
    assert stats["max_inflight"] >= 2, stats   # batches overlapped on the device
    assert stats["max_batch"] >= 2, stats
    for j in jobs:
        i = int(pick[j.jid])
        assert j.result["status"] == 0
        assert result_digest(j.result, cap) == want[i], f"job {j.jid} (pool trace {i}) differs from the oracle"
