"""Helpers shared by the GPU tests: run the CUDA path, compare with the oracle, sample big traces."""
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


def sampled_check(tr, got: dict, n_blocks: int = 16, n_units: int = 1500, seed: int = 0) -> list[str]:
    """Check a full-size GPU result on samples the oracle computes one by one.

    Intra-block races and redundant barriers of a block depend only on that
    block's records; inter-block races of a global unit only on the records of
    that unit; the divergence list only on the barrier counts."""
    rng = np.random.default_rng(seed)
    bad = []
    ev = tr.events
    blocks = rng.choice(tr.n_blocks, size=min(n_blocks, tr.n_blocks), replace=False)
    bsel = np.isin(ev[:, 2], blocks)
    want = oracle.check(sub_trace(tr, bsel))
    if want["status"] != 0:
        return [f"oracle status {want['status']}"]
    g = got["races"]
    gi = g[(g["scope"] == 0) & np.isin(g["block"], blocks)]
    wi = want["races"][want["races"]["scope"] == 0]
    if not (len(gi) == len(wi) and all(np.array_equal(gi[f], wi[f]) for f in g.dtype.names)):
        bad.append(f"intra races of sampled blocks differ ({len(gi)} vs {len(wi)})")
    gr = got["redundant"][np.isin(got["redundant"]["block"], blocks)]
    wr = want["redundant"][np.isin(want["redundant"]["block"], blocks)]
    if not np.array_equal(gr, wr):
        bad.append(f"redundant barriers of sampled blocks differ ({len(gr)} vs {len(wr)})")
    # divergence depends on the counts alone
    empty = tracegen.Trace(np.zeros((0, 4), np.uint32), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                           tr.shared_units, tr.global_units, tr.max_barriers)
    if not np.array_equal(got["divergence"], oracle.check(empty)["divergence"]):
        bad.append("divergence list differs")
    # inter-block races on sampled global units (half of them units that do race)
    glob = ((ev[:, 3] >> 30) & 1) == 1
    if glob.any():
        inter = g[g["scope"] == 1]
        racing = inter["unit"]
        gunits = np.unique(ev[glob, 0])
        pick = rng.choice(gunits, size=min(n_units, len(gunits)), replace=False)
        if len(racing):
            pick = np.union1d(pick, rng.choice(racing, size=min(n_units, len(racing)), replace=False))
        usel = glob & np.isin(ev[:, 0], pick)
        w2 = oracle.check(sub_trace(tr, usel))
        wx = w2["races"][w2["races"]["scope"] == 1]
        gx = inter[np.isin(inter["unit"], pick)]
        if not (len(gx) == len(wx) and all(np.array_equal(gx[f], wx[f]) for f in g.dtype.names)):
            bad.append(f"inter races of sampled units differ ({len(gx)} vs {len(wx)})")
    return bad
