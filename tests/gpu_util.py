"""Helpers shared by the GPU tests: run the CUDA path, compare with the oracle, digest big results."""
from __future__ import annotations

import numpy as np

import oracle
import tracegen

_checkers = {}


def checker(**kw):
    from paper_1905_01833_gb300 import simulee
    key = tuple(sorted(kw.items()))
    if key not in _checkers:
        _checkers[key] = simulee.Checker(0, **kw)
    return _checkers[key]


def gpu_check(tr, races_cap=None, **kw):
    """Check a host trace on the GPU. Large traces get a bounded race list (4M records)."""
    from paper_1905_01833_gb300 import simulee
    if races_cap is None and tr.n_events > 2_000_000:
        races_cap = 4_000_000
    return checker(**kw).check(simulee.to_device(tr), races_cap=races_cap)


def diff(got: dict, want: dict) -> list[str]:
    """Field-by-field differences between a GPU result and an oracle result (empty = identical)."""
    out = []
    for k in ("status", "bad_kind", "bad_index"):
        if int(got[k]) != int(want[k]):
            out.append(f"{k}: gpu {got[k]} oracle {want[k]}")
    if want["status"] != 0:
        return out
    for k in ("races", "divergence", "redundant", "grid_redundant"):
        g, w = got[k], want[k]
        if len(g) != len(w):
            out.append(f"{k}: gpu {len(g)} records, oracle {len(w)}")
            continue
        if g.dtype.names:
            neq = np.zeros(len(g), dtype=bool)
            for f in g.dtype.names:
                neq |= g[f] != w[f]
        else:
            neq = g != w
        if neq.any():
            i = int(np.argmax(neq))
            out.append(f"{k}: first difference at {i}: gpu {g[i]} oracle {w[i]}")
    return out


def sub_trace(tr, mask: np.ndarray):
    """The records selected by mask, same dimensions and barrier counts (order kept)."""
    return tracegen.Trace(tr.events[mask].copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                          tr.shared_units, tr.global_units, tr.max_barriers, tr.flags)


def result_digest(res: dict, races_cap: int) -> str:
    """Digest of a result: status, counts and list bytes, the race list up to races_cap (what an output of
    that capacity holds; a truncated GPU list compares as its prefix plus the true count)."""
    import hashlib
    nr = int(res["n_races"]) if "n_races" in res else len(res["races"])
    status = int(res["status"])
    if status == 4 and nr > races_cap:
        status = 0
    h = hashlib.sha256()
    h.update(np.array([status, int(res["bad_kind"]), int(res["bad_index"]), nr, len(res["divergence"]),
                       len(res["redundant"]), len(res["grid_redundant"])], dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(res["races"][:races_cap]).tobytes())
    for k in ("divergence", "redundant", "grid_redundant"):
        h.update(np.ascontiguousarray(res[k]).tobytes())
    return h.hexdigest()


def make_trace(recipe):
    """A trace from a recipe tuple: ("c2",), ("c4",), ("c3", i, n, block_threads, epochs, seed) or
    ("c5", i, size)."""
    kind = recipe[0]
    if kind == "c2":
        return tracegen.c2()
    if kind == "c4":
        return tracegen.c4()
    if kind == "c3":
        _, i, n, bs, ep, seed = recipe
        return tracegen.c3_trace(i, n, bs, ep, seed=seed)
    if kind == "c5":
        return tracegen.c5_member(recipe[1], recipe[2])
    raise ValueError(recipe)


def oracle_digest(job):
    """(key, records, digest) of the oracle's result on a recipe's trace; runs in a spawned process."""
    key, recipe, races_cap = job
    tr = make_trace(recipe)
    res = oracle.check(tr)
    return key, tr.n_events, result_digest(res, races_cap)


def oracle_digests_async(jobs, processes=None):
    """Start the oracle on many recipes in spawned processes (largest first); returns (pool, async result)."""
    import multiprocessing as mp
    import os
    procs = processes or len(os.sched_getaffinity(0))
    pool = mp.get_context("spawn").Pool(min(procs, max(1, len(jobs))))
    return pool, pool.map_async(oracle_digest, jobs, chunksize=1)
