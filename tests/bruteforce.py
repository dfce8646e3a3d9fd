"""Exhaustive all-pairs checker for tiny traces (pure Python, O(n^2)).

Independent of the C oracle: it does no grouping and no sorting of groups; it
looks at every pair of records and applies the definitions directly
(Theorem 1 without warp refinements, the atomic rule, the inter-block rule for
global memory, the one-barrier-at-a-time redundancy test of Algorithm 5 and the
barrier-count divergence rule of Algorithm 4).

With flag WARP_AWARE (a statement word per record) it applies Theorem 1's
warp clauses: two accesses of one warp (same block, same tid / 32) race only
when both are plain writes with the same statement id, or when either carries
the diverged bit.

With flag PAPER_ORDER it replays Algorithm 3's visit-order counters instead of
using epochs: per (space, block, unit) a counter starts at 0, an access takes
the counter's value, and the barrier at the end of an epoch bumps the counter
when the unit was accessed in that epoch. Pairs of one block then race at
equal counter values, pairs of different blocks on a global unit as well, and
two accesses at consecutive counter values make the barrier that bumped the
counter between them needed.
"""
from __future__ import annotations

import numpy as np

R, W, A = 0, 1, 2


DIVERGED = 0x80000000


def _decode(ev, stmt=None):
    out = []
    for i, w in enumerate(np.asarray(ev, dtype=np.uint64).reshape(-1, 4)):
        w = [int(x) for x in w]
        out.append(dict(i=i, unit=w[0], vo=w[1], block=w[2], tid=w[3] & 0xFFFF, epoch=(w[3] >> 16) & 0xFFF,
                        act=(w[3] >> 28) & 3, space=(w[3] >> 30) & 1, reserved=w[3] >> 31,
                        stmt=None if stmt is None else int(stmt[i])))
    return out


def _conflict(p, q, idp, idq):
    if idp == idq:
        return False
    mp, mq = p["act"] in (W, A), q["act"] in (W, A)
    if not (mp or mq):
        return False
    if p["act"] == A and q["act"] == A:
        return False
    if p["stmt"] is not None and p["block"] == q["block"] and p["tid"] // 32 == q["tid"] // 32:
        same_statement_writes = (p["act"] == W and q["act"] == W and
                                 (p["stmt"] & ~DIVERGED) == (q["stmt"] & ~DIVERGED))
        diverged = bool(p["stmt"] & DIVERGED) or bool(q["stmt"] & DIVERGED)
        if not (same_statement_writes or diverged):
            return False
    return True


def brute(trace) -> dict:
    nb, bt = trace.n_blocks, trace.block_threads
    counts = [int(c) for c in trace.barrier_counts]
    warp_aware = bool(getattr(trace, "flags", 0) & 2)
    recs = _decode(trace.events, getattr(trace, "stmt", None) if warp_aware else None)
    unsorted = bool(getattr(trace, "flags", 0) & 1)
    res = dict(status=0, bad_kind=0, bad_index=0, races=[], divergence=[], redundant=[], grid_redundant=[])
    for t, c in enumerate(counts):
        if c > trace.max_barriers:
            res.update(status=2, bad_kind=1, bad_index=t)
            return res
    for r in recs:
        ok = r["block"] < nb and r["tid"] < bt and r["act"] != 3 and r["reserved"] == 0
        ok = ok and r["unit"] < (trace.global_units if r["space"] else trace.shared_units)
        if ok and r["epoch"] > counts[r["block"] * bt + r["tid"]]:
            ok = False
        if not unsorted and r["i"] > 0 and r["vo"] <= recs[r["i"] - 1]["vo"]:
            ok = False
        if not ok:
            res.update(status=2, bad_kind=0, bad_index=r["i"])
            return res

    def order(r):
        return (r["vo"], r["i"])

    paper = bool(getattr(trace, "flags", 0) & 4)
    if paper:   # Algorithm 3: replay the counters epoch by epoch
        touched = {}
        for r in recs:
            touched.setdefault((r["space"], r["block"], r["unit"]), set()).add(r["epoch"])
        counter_at = {}
        for key, eps in touched.items():
            c, vals = 0, {}
            for e in range(max(eps) + 1):
                vals[e] = c
                if e in eps:      # the barrier ending epoch e bumps a unit accessed in epoch e
                    c += 1
            counter_at[key] = vals
        for r in recs:
            r["pvo"] = counter_at[(r["space"], r["block"], r["unit"])][r["epoch"]]

    best = {}
    nonred = set()
    for a in recs:
        for b in recs:
            if a is b or order(a) >= order(b):
                continue
            p, q = a, b        # p earlier than q
            gp, gq = p["block"] * bt + p["tid"], q["block"] * bt + q["tid"]
            if p["unit"] != q["unit"] or p["space"] != q["space"]:
                continue
            cls = 0 if (p["act"] in (W, A) and q["act"] in (W, A)) else 1
            if p["block"] == q["block"]:
                if p["epoch"] == q["epoch"] and _conflict(p, q, gp, gq):
                    key = (p["space"], 0, p["block"], p["epoch"], p["unit"], cls)
                    cand = (order(q), order(p), p, q)
                    if key not in best or cand[:2] < best[key][:2]:
                        best[key] = cand
                lo, hi = (p, q) if p["epoch"] < q["epoch"] else (q, p)
                if paper:
                    # consecutive counter values: the barrier ending lo's epoch made the step
                    if hi["pvo"] == lo["pvo"] + 1 and _conflict(lo, hi, gp, gq):
                        nonred.add((p["block"], lo["epoch"]))
                elif hi["epoch"] == lo["epoch"] + 1 and _conflict(lo, hi, gp, gq):
                    nonred.add((p["block"], lo["epoch"]))
            elif p["space"] == 1 and (not paper or p["pvo"] == q["pvo"]) and _conflict(p, q, p["block"], q["block"]):
                key = (1, 1, 0xFFFFFFFF, q["pvo"] if paper else 0xFFFFFFFF, p["unit"], cls)
                cand = (order(q), order(p), p, q)
                if key not in best or cand[:2] < best[key][:2]:
                    best[key] = cand
    races = []
    for key in sorted(best):
        _, _, p, q = best[key]
        space, scope, block, epoch, unit, cls = key
        races.append((space, scope, cls, block, epoch, unit, p["vo"], q["vo"],
                      p["block"] * bt + p["tid"], q["block"] * bt + q["tid"]))
    res["races"] = races

    divs, maxc = [], []
    for b in range(nb):
        cs = counts[b * bt:(b + 1) * bt]
        maxc.append(max(cs))
        if min(cs) != max(cs):
            divs.append((b, min(cs), max(cs), cs.index(min(cs))))
    res["divergence"] = divs
    bars = [(b, k) for b in range(nb) for k in range(maxc[b]) if (b, k) not in nonred]
    res["redundant"] = bars
    gmax = max(maxc) if maxc else 0
    res["grid_redundant"] = [k for k in range(gmax)
                             if all((b, k) not in nonred for b in range(nb) if maxc[b] > k)]
    return res


def as_tuples(out: dict) -> dict:
    """Convert a structured-array result (oracle or GPU) to the brute-force tuple form."""
    r = out["races"]
    races = [(int(x["space"]), int(x["scope"]), int(x["cls"]), int(x["block"]), int(x["epoch"]), int(x["unit"]),
              int(x["vo_first"]), int(x["vo_second"]), int(x["gtid_first"]), int(x["gtid_second"])) for x in r]
    divs = [tuple(int(v) for v in x) for x in out["divergence"]]
    bars = [tuple(int(v) for v in x) for x in out["redundant"]]
    grid = [int(x) for x in out["grid_redundant"]]
    return dict(status=out["status"], bad_kind=out["bad_kind"], bad_index=out["bad_index"],
                races=races, divergence=divs, redundant=bars, grid_redundant=grid)
