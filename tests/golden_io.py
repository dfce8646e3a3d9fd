"""Reader for the worked-example fixtures under tests/golden/."""
from __future__ import annotations

import os

import tracegen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_ACT = {"R": 0, "W": 1, "A": 2}
_SP = {"S": 0, "G": 1}
_SCOPE = {"intra": 0, "inter": 1}
_CLS = {"WW": 0, "RW": 1}


def load(name: str):
    """Return a list of (trace, expected) pairs, one per '---'-separated section."""
    text = open(os.path.join(GOLDEN, name)).read()
    out = []
    for sec in text.split("\n---"):
        dims, counts, recs = {}, [], []
        exp = dict(races=[], redundant=None, divergence=None)
        for line in sec.splitlines():
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "dims":
                dims = {k: int(v) for k, v in (t.split("=") for t in tok[1:])}
            elif tok[0] == "counts":
                counts = [int(x) for x in tok[1:]]
            elif tok[0] == "rec":
                blk, tid, ep, unit = (int(x) for x in tok[1:5])
                recs.append((unit, len(recs), blk, tid, ep, _ACT[tok[5]], _SP[tok[6]]))
            elif tok[0] == "expect":
                what, rest = tok[1], tok[2:]
                if what == "races" and rest:
                    vals = [_SP[rest[0]], _SCOPE[rest[1]], _CLS[rest[2]]] + [int(x) for x in rest[3:]]
                    exp["races"].append(tuple(vals))
                elif what == "redundant":
                    exp["redundant"] = [tuple(int(v) for v in x.split(":")) for x in rest]
                elif what == "divergence":
                    exp["divergence"] = [tuple(int(v) for v in x.split(":")) for x in rest]
        b = tracegen.Builder(dims["n_blocks"], dims["block_threads"], dims["shared_units"], dims["global_units"])
        for r in recs:
            b.access(r[2], r[3], r[4], r[0], r[5], r[6])
        b.counts[:] = counts
        tr = b.trace(max_barriers=dims["max_barriers"])
        out.append((tr, exp))
    return out


def race_tuples(out):
    """(space, scope, cls, block, epoch, unit, vo_first, vo_second, gtid_first, gtid_second) in output order."""
    return [(int(x["space"]), int(x["scope"]), int(x["cls"]), int(x["block"]), int(x["epoch"]), int(x["unit"]),
             int(x["vo_first"]), int(x["vo_second"]), int(x["gtid_first"]), int(x["gtid_second"]))
            for x in out["races"]]
