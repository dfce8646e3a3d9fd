"""Hand-built traces with closed-form expected results.

Each builder returns (trace, expect). `expect` holds what the definitions fix
for that trace, derived by hand in the builder's docstring:
    races:       set of (space, scope, cls, block, epoch, unit, gtid_first, gtid_second)
    redundant:   list of (block, barrier)
    divergence:  list of (block, min, max, first_min_tid)
    grid:        list of barrier indices
Visit orders of the lowest pairs are checked separately where stated
(`vo_order`: the writer/reader roles fix which access comes first).
"""
from __future__ import annotations

import tracegen
from tracegen import ATOMIC, GLOBAL, READ, SHARED, WRITE, Builder

RW, WW = 1, 0


def tree_reduction(bt: int = 64, remove_after: int | None = None):
    """Shared-memory tree reduction over sh[0..bt).

    Epoch 0: every thread t writes sh[t]. Step i = 1..L (s_i = bt >> i): threads
    t < s_i read sh[t] and sh[t+s_i], then write sh[t]; a barrier follows every
    epoch, so counts = L and nothing races. Every barrier k is needed: epoch k+1
    reads sh[t + s_{k+1}], written in epoch k by thread t + s_{k+1}.

    Without the barrier after epoch j (epochs after j relabelled one lower), the
    merged epoch j holds the writes of step j (s_0 = bt) and the reads of step
    j+1: unit u in [s_{j+1}, s_j) is written by thread u and read by thread
    u - s_{j+1}: exactly one RW race per such unit, writer first. There is no
    WW race: a unit u < s_{j+1} is written in both steps by thread u itself.
    Every remaining barrier is still needed, for the reason above.
    """
    L = bt.bit_length() - 1
    b = Builder(1, bt, bt)
    for e in range(L + 1):
        lab = e if remove_after is None or e <= remove_after else e - 1
        if e == 0:
            for t in range(bt):
                b.access(0, t, lab, t, WRITE)
        else:
            s = bt >> e
            for t in range(s):
                b.access(0, t, lab, t, READ)
            for t in range(s):
                b.access(0, t, lab, t + s, READ)
            for t in range(s):
                b.access(0, t, lab, t, WRITE)
    b.set_counts(L if remove_after is None else L - 1)
    tr = b.trace()
    if remove_after is None:
        return tr, dict(races=set(), redundant=[], divergence=[], grid=[])
    j = remove_after
    sj = bt >> j if j > 0 else bt
    sj1 = bt >> (j + 1)
    races = {(SHARED, 0, RW, 0, j, u, u, u - sj1) for u in range(sj1, sj)}
    return tr, dict(races=races, redundant=[], divergence=[], grid=[], vo_order="writer_first")


def transpose(with_barrier: bool = True):
    """32x8 threads move a 32x32 tile (pitch 33) through shared memory.

    Thread (tx, ty), tid = tx + 32*ty, writes tile[ty+8j][tx] (j = 0..3), then
    reads tile[tx][ty+8j]. With a barrier between the phases nothing races and
    the barrier is needed (the reader of unit (r,c), r != c, is another thread).
    Without it (one epoch): unit r*33+c with r != c is written by thread
    (c, r mod 8) and read by thread (r, c mod 8), different threads, so exactly
    one RW race per off-diagonal unit (992 units); diagonal units are written
    and read by the same thread.
    """
    b = Builder(1, 256, 32 * 33)
    e1 = 1 if with_barrier else 0
    for j in range(4):
        for t in range(256):
            tx, ty = t % 32, t // 32
            b.access(0, t, 0, (ty + 8 * j) * 33 + tx, WRITE)
    for j in range(4):
        for t in range(256):
            tx, ty = t % 32, t // 32
            b.access(0, t, e1, tx * 33 + ty + 8 * j, READ)
    b.set_counts(1 if with_barrier else 0)
    tr = b.trace()
    if with_barrier:
        return tr, dict(races=set(), redundant=[], divergence=[], grid=[])
    races = set()
    for r in range(32):
        for c in range(32):
            if r != c:
                races.add((SHARED, 0, RW, 0, 0, r * 33 + c, c + 32 * (r % 8), r + 32 * (c % 8)))
    return tr, dict(races=races, redundant=[], divergence=[], grid=[], vo_order="writer_first")


def atomic_counters(n_blocks: int = 3, bt: int = 16, peek: bool = False):
    """Every thread of every block does one atomic on global counter (t mod 4).

    Atomics never race with atomics, so there is nothing to report. With `peek`,
    thread 0 of block 0 then reads counter 0 plainly (last access). Intra-block:
    the lowest RW pair on unit 0 of block 0 is (atomic of thread 4, the read) -
    thread 0's own atomic is the same owner. Inter-block: (the first atomic on
    unit 0 from block 1, i.e. thread 0 of block 1, the read).
    """
    b = Builder(n_blocks, bt, 0, 4)
    for blk in range(n_blocks):
        for t in range(bt):
            b.access(blk, t, 0, t % 4, ATOMIC, GLOBAL)
    if peek:
        b.access(0, 0, 0, 0, READ, GLOBAL)
    b.set_counts(0)
    tr = b.trace()
    races = set()
    if peek:
        races = {(GLOBAL, 0, RW, 0, 0, 0, 4, 0),
                 (GLOBAL, 1, RW, 0xFFFFFFFF, 0xFFFFFFFF, 0, bt * 1 + 0, 0)}
    return tr, dict(races=races, redundant=[], divergence=[], grid=[])


def homography(bt: int = 32, epochs: int = 4):
    """Thread-private shared arrays s_median[tid], s_idx[tid] (Sec. 2, arrayfire).

    Each thread reads and writes only its own two units in every epoch, so no
    pair of distinct threads ever shares a unit: no races, and every barrier is
    redundant in the block and therefore grid-wide.
    """
    b = Builder(1, bt, 2 * bt)
    for e in range(epochs):
        for t in range(bt):
            b.access(0, t, e, t, WRITE)
        for t in range(bt):
            b.access(0, t, e, bt + t, WRITE)
        for t in range(bt):
            b.access(0, t, e, t, READ)
    b.set_counts(epochs - 1)
    tr = b.trace()
    return tr, dict(races=set(), redundant=[(0, k) for k in range(epochs - 1)], divergence=[],
                    grid=list(range(epochs - 1)))


def thundersvm(bt: int = 32, fixed: bool = False):
    """WW shape of the thundersvm fix (Sec. 2): a branch writes f[t] and a block
    reduction then writes the same array without a barrier in between.

    Thread t writes f[t]; then thread t >= bt/2 writes f[t - bt/2]. Without the
    barrier, unit u < bt/2 is written by thread u and then by thread u + bt/2:
    one WW race per such unit. With the fix (a barrier between the two), there
    is no race and the barrier is needed.
    """
    b = Builder(1, bt, bt)
    for t in range(bt):
        b.access(0, t, 0, t, WRITE)
    e = 1 if fixed else 0
    for t in range(bt // 2, bt):
        b.access(0, t, e, t - bt // 2, WRITE)
    b.set_counts(1 if fixed else 0)
    tr = b.trace()
    if fixed:
        return tr, dict(races=set(), redundant=[], divergence=[], grid=[])
    races = {(SHARED, 0, WW, 0, 0, u, u, u + bt // 2) for u in range(bt // 2)}
    return tr, dict(races=races, redundant=[], divergence=[], grid=[], vo_order="writer_first")


def divergent(n_blocks: int = 4, bt: int = 8, bad_block: int = 2, bad_tid: int = 5):
    """One thread of one block skips the block's only barrier (Sec. 2, arrayfire
    nearest_neighbour: a barrier inside a branch). Its count is 0 while the
    others' are 1: only that block is listed, as (block, 0, 1, bad_tid)."""
    b = Builder(n_blocks, bt, 2 * bt)
    for blk in range(n_blocks):
        for e in range(2):
            for t in range(bt):
                lab = 0 if (blk == bad_block and t == bad_tid) else e
                b.access(blk, t, lab, e * bt + t, WRITE)
    b.set_counts(1)
    b.set_counts(0, bad_block, bad_tid)
    tr = b.trace()
    return tr, dict(divergence=[(bad_block, 0, 1, bad_tid)])


ALL = {
    "tree_barriers": lambda: tree_reduction(64),
    "tree_no_barrier_0": lambda: tree_reduction(64, 0),
    "tree_no_barrier_2": lambda: tree_reduction(64, 2),
    "tree_no_barrier_last": lambda: tree_reduction(64, 5),
    "transpose_barrier": lambda: transpose(True),
    "transpose_no_barrier": lambda: transpose(False),
    "atomics": lambda: atomic_counters(3, 16, False),
    "atomics_peek": lambda: atomic_counters(3, 16, True),
    "homography": lambda: homography(),
    "thundersvm": lambda: thundersvm(fixed=False),
    "thundersvm_fixed": lambda: thundersvm(fixed=True),
    "divergent": lambda: divergent(),
}


def _valid_base():
    b = Builder(2, 4, 8, 8)
    for blk in range(2):
        for t in range(4):
            b.access(blk, t, 0, t, WRITE)
            b.access(blk, t, 1, (t + 1) % 4, READ, GLOBAL)
    b.set_counts(1)
    return b.trace()


BAD_RECORDS = [("block", 3), ("tid", 5), ("action3", 0), ("reserved", 7), ("shared_unit", 2),
               ("global_unit", 9), ("epoch", 4), ("vo_equal", 6), ("vo_down", 11)]


def bad_record(what: str, idx: int):
    """A valid 16-record trace with record `idx` broken in one field (and record 14
    broken too, later, so only the first bad index may be reported).
    Expected status: EBADTRACE (2), kind 0 (a record), index idx."""
    tr = _valid_base()
    ev = tr.events
    w3 = int(ev[idx, 3])
    if what == "block":
        ev[idx, 2] = 2
    elif what == "tid":
        ev[idx, 3] = (w3 & ~0xFFFF) | 4
    elif what == "action3":
        ev[idx, 3] = w3 | (3 << 28)
    elif what == "reserved":
        ev[idx, 3] = w3 | (1 << 31)
    elif what == "shared_unit":
        ev[idx, 3] = w3 & ~(1 << 30)
        ev[idx, 0] = 8
    elif what == "global_unit":
        ev[idx, 3] = w3 | (1 << 30)
        ev[idx, 0] = 8
    elif what == "epoch":
        ev[idx, 3] = (w3 & ~(0xFFF << 16)) | (2 << 16)
    elif what == "vo_equal":
        ev[idx, 1] = ev[idx - 1, 1]
    elif what == "vo_down":
        ev[idx, 1] = 0
    ev[14, 2] = 9
    return tr, (2, 0, idx)


def bad_count():
    """Counts are checked before records: a bad record 0 and bad counts at
    threads 5 and 6 give kind 1 (a count), index 5."""
    tr = _valid_base()
    tr.events[0, 2] = 7
    tr.barrier_counts[5] = tr.max_barriers + 1
    tr.barrier_counts[6] = tr.max_barriers + 3
    return tr, (2, 1, 5)


def race_keys(out) -> set:
    r = out["races"]
    return {(int(x["space"]), int(x["scope"]), int(x["cls"]), int(x["block"]), int(x["epoch"]), int(x["unit"]),
             int(x["gtid_first"]), int(x["gtid_second"])) for x in r}


def check_expect(out, expect) -> list[str]:
    """Return the list of mismatches between a result and a closed-form expectation."""
    bad = []
    if out["status"] != 0:
        return [f"status {out['status']}"]
    if "races" in expect and race_keys(out) != expect["races"]:
        got = race_keys(out)
        bad.append(f"races: missing {sorted(expect['races'] - got)[:4]} extra {sorted(got - expect['races'])[:4]}")
    if "redundant" in expect:
        got = [tuple(int(v) for v in x) for x in out["redundant"]]
        if got != expect["redundant"]:
            bad.append(f"redundant {got} != {expect['redundant']}")
    if "divergence" in expect:
        got = [tuple(int(v) for v in x) for x in out["divergence"]]
        if got != expect["divergence"]:
            bad.append(f"divergence {got} != {expect['divergence']}")
    if "grid" in expect:
        got = [int(x) for x in out["grid_redundant"]]
        if got != expect["grid"]:
            bad.append(f"grid {got} != {expect['grid']}")
    if expect.get("vo_order") == "writer_first":
        for x in out["races"]:
            if not x["vo_first"] < x["vo_second"]:
                bad.append("lowest pair not ordered")
                break
    return bad


def tracegen_module():
    return tracegen
