"""Seeded synthetic access-record traces.

This module only synthesises inputs for the synchronization check: 16-byte
access records plus per-thread barrier counts. It holds none of the
detection arithmetic; the CPU oracle and the CUDA path both consume what it
produces and neither is imported here.

Record layout (four little-endian uint32 words per record):
    w0 unit, w1 visit_order, w2 block,
    w3 = tid[0:16] | epoch[16:28] | action[28:30] | space[30] | reserved[31]
with action 0 read / 1 write / 2 atomic and space 0 shared / 1 global.

The bulk generators are C (``tracegen.c``), compiled on first use with gcc.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

READ, WRITE, ATOMIC = 0, 1, 2
SHARED, GLOBAL = 0, 1
UNSORTED = 1  # trace flag: visit orders are not increasing in record order
WARP_AWARE = 2  # trace flag: records carry statement words (Theorem 1's warp refinements apply)
PAPER_ORDER = 4  # trace flag: the paper's visit-order counters (Algorithm 3) group the tuples
DIVERGED = 0x80000000  # statement-word bit: the access came after the thread's warp diverged

DEFAULT_SEED = 1905018330

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tracegen.c")
_SO = os.path.join(_HERE, "libtracegen.so")
_lock = threading.Lock()
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile tracegen.c into libtracegen.so (host code, any architecture)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _PatternParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_blocks", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("n_epochs", ctypes.c_uint32),
        ("shared_units", ctypes.c_uint32),
        ("global_units", ctypes.c_uint32),
        ("removed_p", ctypes.c_double),
        ("atomic_p", ctypes.c_double),
        ("peek_p", ctypes.c_double),
        ("stray_p", ctypes.c_double),
    ]


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.tg_strided.restype = ctypes.c_uint64
            lib.tg_strided.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_double, ctypes.c_double, vp, vp]
            lib.tg_pattern.restype = ctypes.c_uint64
            lib.tg_pattern.argtypes = [ctypes.POINTER(_PatternParams), vp, vp]
            lib.tg_barrier.restype = ctypes.c_uint64
            lib.tg_barrier.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.c_double, vp, vp, vp]
            _lib_handle = lib
    return _lib_handle


@dataclasses.dataclass
class Trace:
    """A trace: records, per-thread barrier counts and the dimensions they live in."""
    events: np.ndarray            # uint32 (n, 4)
    barrier_counts: np.ndarray    # uint32 (n_blocks * block_threads,)
    n_blocks: int
    block_threads: int
    shared_units: int
    global_units: int
    max_barriers: int
    flags: int = 0
    meta: dict = dataclasses.field(default_factory=dict)
    stmt: np.ndarray | None = None   # warp-aware traces: per record, statement id | DIVERGED

    @property
    def n_events(self) -> int:
        return int(self.events.shape[0])


def pack(unit, vo, block, tid, epoch, action, space):
    """Pack record fields (scalars or arrays) into an (n, 4) uint32 array."""
    unit = np.asarray(unit, dtype=np.uint64)
    w3 = (np.asarray(tid, dtype=np.uint64) & 0xFFFF) | ((np.asarray(epoch, dtype=np.uint64) & 0xFFF) << 16) \
        | ((np.asarray(action, dtype=np.uint64) & 3) << 28) | ((np.asarray(space, dtype=np.uint64) & 1) << 30)
    out = np.stack(np.broadcast_arrays(unit, np.asarray(vo, dtype=np.uint64),
                                       np.asarray(block, dtype=np.uint64), w3), axis=-1)
    return np.ascontiguousarray(out.astype(np.uint32).reshape(-1, 4))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def strided(seed: int = DEFAULT_SEED, n_threads: int = 256, n_epochs: int = 8, per_thread: int = 16,
            shared_units: int = 12288, write_p: float = 0.25, redirect_p: float = 0.001) -> Trace:
    """One block; per epoch a stride s in {1,2,32}; thread t touches (t*s+k) mod units."""
    lib = _lib()
    n = lib.tg_strided(seed, n_threads, n_epochs, per_thread, shared_units, write_p, redirect_p, None, None)
    ev = np.empty((n, 4), dtype=np.uint32)
    counts = np.empty(n_threads, dtype=np.uint32)
    lib.tg_strided(seed, n_threads, n_epochs, per_thread, shared_units, write_p, redirect_p, _ptr(ev), _ptr(counts))
    return Trace(ev, counts, 1, n_threads, shared_units, 0, n_epochs - 1,
                 meta=dict(kind="strided", seed=seed))


def pattern(seed: int = DEFAULT_SEED, n_blocks: int = 1024, block_threads: int = 256, n_epochs: int = 32,
            shared_units: int = 12288, global_units: int = 1 << 26, removed_p: float = 0.10,
            atomic_p: float = 0.02, peek_p: float = 0.01, stray_p: float = 0.001) -> Trace:
    """Grid of tree-reduction / tiled-transpose blocks over shared and global memory."""
    lib = _lib()
    pp = _PatternParams(seed, n_blocks, block_threads, n_epochs, shared_units, global_units,
                        removed_p, atomic_p, peek_p, stray_p)
    n = lib.tg_pattern(ctypes.byref(pp), None, None)
    if n == 0:
        raise ValueError("pattern: dimensions do not fit the access patterns")
    ev = np.empty((n, 4), dtype=np.uint32)
    counts = np.empty(n_blocks * block_threads, dtype=np.uint32)
    lib.tg_pattern(ctypes.byref(pp), _ptr(ev), _ptr(counts))
    return Trace(ev, counts, n_blocks, block_threads, shared_units, global_units, n_epochs - 1,
                 meta=dict(kind="pattern", seed=seed))


def redundant_set(seed: int, n_barriers: int, count: int) -> int:
    """Bit mask of `count` distinct barrier indices in [0, n_barriers), seeded."""
    rng = np.random.default_rng(seed ^ 0x5EED)
    chosen = rng.choice(n_barriers, size=min(count, n_barriers), replace=False)
    mask = 0
    for k in chosen:
        mask |= 1 << int(k)
    return mask


def barrier(seed: int = DEFAULT_SEED, n_blocks: int = 1024, block_threads: int = 1024, n_epochs: int = 64,
            shared_units: int = 8192, per_thread: int = 4, redundant_fraction: float = 0.2,
            redirect_p: float = 1e-5, diverge_p: float = 0.01) -> Trace:
    """Barrier-analysis family: known redundant set and known divergent blocks."""
    lib = _lib()
    nbar = n_epochs - 1
    mask = redundant_set(seed, nbar, int(round(redundant_fraction * nbar)))
    args = (seed, n_blocks, block_threads, n_epochs, shared_units, per_thread, mask, redirect_p, diverge_p)
    n = lib.tg_barrier(*args, None, None, None)
    if n == 0:
        raise ValueError("barrier: dimensions do not fit")
    ev = np.empty((n, 4), dtype=np.uint32)
    counts = np.empty(n_blocks * block_threads, dtype=np.uint32)
    div = np.empty(n_blocks, dtype=np.uint8)
    lib.tg_barrier(*args, _ptr(ev), _ptr(counts), _ptr(div))
    return Trace(ev, counts, n_blocks, block_threads, shared_units, 0, n_epochs - 1,
                 meta=dict(kind="barrier", seed=seed, redundant_mask=mask,
                           divergent_blocks=np.nonzero(div)[0].astype(np.uint32)))


# --- the five named workloads --------------------------------------------------

def c1(seed: int = DEFAULT_SEED) -> Trace:
    """1 block x 256 threads, 8 epochs, 12288 shared units, 16 accesses/thread/epoch (32,768 records)."""
    return strided(seed, 256, 8, 16, 12288, 0.25, 0.001)


def c2(seed: int = DEFAULT_SEED, n_blocks: int = 1024) -> Trace:
    """1024 blocks x 256 threads, 32 epochs, 12288 shared + 2^26 global units (~6e7 records)."""
    return pattern(seed, n_blocks, 256, 32, 12288, 1 << 26)


def c4(seed: int = DEFAULT_SEED, n_blocks: int = 1024) -> Trace:
    """1024 blocks x 1024 threads, 64 epochs, 4 accesses/thread/epoch (2^28 records)."""
    return barrier(seed, n_blocks, 1024, 64, 8192, 4)


C3_RECORDS = 600_000_000   # records of the batched workload, all traces together


def c3_sigma(seed: int = DEFAULT_SEED, n_traces: int = 4096, median: float = 1e5, lo: float = 1e3,
             hi: float = 1e7, total: int = C3_RECORDS) -> float:
    """The lognormal sigma whose seeded, clipped size draws sum to `total` records (bisection).

    The draws are exp(ln(median) + sigma * z_i) with the seeded standard normals z_i of c3_sizes,
    clipped to [lo, hi] and truncated to integers; their sum increases with sigma over the bracket."""
    z = np.random.default_rng(seed).standard_normal(n_traces)

    def tot(s):
        return int(np.clip(np.exp(np.log(median) + s * z), lo, hi).astype(np.int64).sum())
    a, b = 0.3, 3.0
    if not (tot(a) <= total <= tot(b)):
        raise ValueError("c3_sigma: total out of reach")
    for _ in range(64):
        m = 0.5 * (a + b)
        if tot(m) < total:
            a = m
        else:
            b = m
    return b


def c3_sizes(seed: int = DEFAULT_SEED, n_traces: int = 4096, median: float = 1e5, sigma: float | None = None,
             lo: float = 1e3, hi: float = 1e7, total: int = C3_RECORDS):
    """Per-trace (records, block size, epochs) for the batched workload. Without an explicit sigma,
    sigma is fitted so that the sizes sum to `total` (c3_sigma)."""
    if sigma is None:
        sigma = c3_sigma(seed, n_traces, median, lo, hi, total)
    rng = np.random.default_rng(seed)
    n = np.clip(np.exp(np.log(median) + sigma * rng.standard_normal(n_traces)), lo, hi)
    bs = rng.choice(np.array([64, 128, 256, 1024]), size=n_traces)
    ep = rng.integers(4, 65, size=n_traces)
    return n.astype(np.int64), bs.astype(np.int64), ep.astype(np.int64)


def c3_trace(i: int, target: int, block_threads: int, n_epochs: int, seed: int = DEFAULT_SEED) -> Trace:
    """One trace of the batched workload: the grid pattern with enough blocks for
    `target` records, cut to its first `target` records in schedule order. The
    block count starts from 8 records per thread per epoch and grows (from the
    records per block of the last attempt) until the pattern holds the target.
    Barrier counts stay those of the full run, so the cut trace is a valid trace
    whose last block ends early (its later epochs are empty)."""
    nb = max(1, int(np.ceil(target / (block_threads * n_epochs * 8))))
    for _ in range(8):
        gu = 1 << int(np.ceil(np.log2(4096 + 2 * 1024 * nb)))
        tr = pattern(seed + 7919 * (i + 1), nb, block_threads, n_epochs, 12288, gu)
        if tr.n_events >= target:
            break
        nb = max(nb + 1, int(np.ceil(1.05 * target * nb / max(tr.n_events, 1))))
    if tr.n_events > target:
        tr.events = np.ascontiguousarray(tr.events[:target])
    tr.meta.update(kind="batch_member", target=int(target))
    return tr


C5_SIZES = (1e4, 1e8)   # record range of the served workload's jobs (log-uniform)


def c5_pool_sizes(n_pool: int = 24) -> np.ndarray:
    """Sizes of the served workload's pool of traces: log-spaced over C5_SIZES."""
    return np.exp(np.linspace(np.log(C5_SIZES[0]), np.log(C5_SIZES[1]), n_pool))


def c5_member(i: int, size: float) -> Trace:
    """Pool trace i of the served workload: even i the grid family (256-thread blocks, 32 epochs,
    about 6e4 records per block), odd i the barrier family (1024-thread blocks, 64 epochs, 4 accesses
    per thread per epoch, 262144 records per block); cut to `size` records in schedule order."""
    if i % 2 == 0:
        nb = max(1, int(round(size / 59600)))
        tr = pattern(100 + i, n_blocks=nb, block_threads=256, n_epochs=32, shared_units=12288,
                     global_units=1 << max(20, int(np.ceil(np.log2(4096 + 2 * 1024 * nb)))))
    else:
        nb = max(1, int(round(size / 262144)))
        tr = barrier(100 + i, n_blocks=nb, block_threads=1024, n_epochs=64, shared_units=8192)
    if tr.n_events > size:
        tr.events = np.ascontiguousarray(tr.events[:int(size)])
    tr.meta.update(kind="serve_member", index=i)
    return tr


# --- tiny random traces (for exhaustive pair checks) ---------------------------

def random_tiny(seed: int, n_events: int | None = None, n_blocks: int | None = None,
                block_threads: int | None = None, max_epochs: int | None = None,
                units: int | None = None, p_global: float = 0.4, p_atomic: float = 0.15,
                p_write: float = 0.35, unsorted: bool = False) -> Trace:
    """A small random trace with valid fields; visit orders increase with random gaps."""
    rng = np.random.default_rng(seed)
    nb = n_blocks or int(rng.integers(1, 5))
    bt = block_threads or int(rng.integers(1, 9))
    me = max_epochs or int(rng.integers(1, 5))
    su = units or int(rng.integers(1, 9))
    gu = units or int(rng.integers(1, 9))
    n = n_events if n_events is not None else int(rng.integers(0, 120))
    counts = rng.integers(0, me, size=nb * bt).astype(np.uint32)
    # most blocks agree on their count; some threads diverge
    for b in range(nb):
        if rng.random() < 0.7:
            counts[b * bt:(b + 1) * bt] = counts[b * bt]
    block = rng.integers(0, nb, size=n)
    tid = rng.integers(0, bt, size=n)
    gt = block * bt + tid
    epoch = (rng.random(n) * (counts[gt].astype(np.float64) + 1)).astype(np.int64)
    epoch = np.minimum(epoch, counts[gt])
    space = (rng.random(n) < p_global).astype(np.int64)
    r = rng.random(n)
    act = np.where(r < p_atomic, ATOMIC, np.where(r < p_atomic + p_write, WRITE, READ))
    unit = np.where(space == 1, rng.integers(0, gu, size=n), rng.integers(0, su, size=n))
    vo = np.cumsum(rng.integers(1, 4, size=n)) if n else np.zeros(0, dtype=np.int64)
    flags = 0
    if unsorted:
        # shuffle record order and let some visit orders collide
        vo = rng.integers(0, max(1, n // 2), size=n)
        flags = UNSORTED
    ev = pack(unit, vo, block, tid, epoch, act, space)
    return Trace(ev, counts, nb, bt, su, gu, me - 1 if me > 1 else 0, flags,
                 meta=dict(kind="random_tiny", seed=seed))


def random_grouped(seed: int, **kw) -> Trace:
    """A random tiny trace reordered into simulator order: records sorted by
    (block, epoch) (stable), visit orders renumbered 0..n-1."""
    tr = random_tiny(seed, unsorted=False, **kw)
    ev = tr.events
    epoch = (ev[:, 3] >> 16) & 0xFFF
    order = np.lexsort((np.arange(len(ev)), epoch, ev[:, 2]))
    ev = np.ascontiguousarray(ev[order])
    ev[:, 1] = np.arange(len(ev), dtype=np.uint32)
    tr.events = ev
    tr.meta["kind"] = "random_grouped"
    return tr


def broadcast(seed: int = DEFAULT_SEED, n_blocks: int = 64, block_threads: int = 256, n_epochs: int = 8,
              reads: int = 1, global_const: bool = True, writers: bool = True) -> Trace:
    """Kernels whose threads share hot units: per epoch every thread reads the epoch's shared broadcast unit
    `reads` times (e mod 4; thread 0 writes it in the epoch before when that epoch is even), adds into one of 32 shared histogram bins
    (eight consecutive threads per bin; a plain write instead of an atomic in every fourth epoch), writes a
    private shared unit and, with `global_const`, reads one global unit that every thread of the grid reads
    (a kernel-wide constant). With `writers`, one thread per block also writes the broadcast unit in epochs
    e = 1 mod 3 and thread 0 of each block writes the global constant in epochs e = 2 mod 5, so the hot
    units' groups hold races. Emission order: block, epoch, slot, thread; visit order = position. Global
    writes of thread t go to its own unit b * block_threads + t (no conflicts)."""
    bt, E = block_threads, n_epochs
    gconst = (1 << 24) - 1
    t = np.arange(bt, dtype=np.int64)
    rng = np.random.default_rng(seed)
    wtid = rng.integers(1, bt, size=n_blocks)   # the block's extra writer of the broadcast unit
    units, blocks, tids, epochs, acts, spaces = [], [], [], [], [], []

    def put(u, b, th, e, a, sp):
        n = len(th)
        units.append(np.broadcast_to(np.asarray(u, dtype=np.int64), (n,)))
        blocks.append(np.full(n, b, dtype=np.int64))
        tids.append(np.asarray(th, dtype=np.int64))
        epochs.append(np.full(n, e, dtype=np.int64))
        acts.append(np.broadcast_to(np.asarray(a, dtype=np.int64), (n,)))
        spaces.append(np.full(n, sp, dtype=np.int64))

    for b in range(n_blocks):
        for e in range(E):
            for _ in range(reads):
                put(e % 4, b, t, e, READ, SHARED)
            if writers and e % 3 == 1:
                put(e % 4, b, [int(wtid[b])], e, WRITE, SHARED)
            put(8 + (t // 8 + e) % 32, b, t, e, WRITE if e % 4 == 3 else ATOMIC, SHARED)
            put(64 + t, b, t, e, WRITE, SHARED)
            if global_const:
                put(gconst, b, t, e, READ, GLOBAL)
            if writers and e % 5 == 2:
                put(gconst, b, [0], e, WRITE, GLOBAL)
            put((b * bt + t) % gconst, b, t, e, WRITE, GLOBAL)
            if e % 2 == 0:
                put((e + 1) % 4, b, [0], e, WRITE, SHARED)
    u = np.concatenate(units)
    ev = pack(u, np.arange(len(u)), np.concatenate(blocks), np.concatenate(tids), np.concatenate(epochs),
              np.concatenate(acts), np.concatenate(spaces))
    counts = np.full(n_blocks * bt, E - 1, dtype=np.uint32)
    return Trace(ev, counts, n_blocks, bt, 4096, 1 << 24, E - 1,
                 meta=dict(kind="broadcast", seed=seed, reads=reads, global_const=global_const, writers=writers))


class Builder:
    """Hand-built traces: records are appended in schedule order (visit order = serial)."""

    def __init__(self, n_blocks: int, block_threads: int, shared_units: int, global_units: int = 0):
        self.nb, self.bt, self.su, self.gu = n_blocks, block_threads, shared_units, global_units
        self.rows: list[tuple] = []
        self.counts = np.zeros(n_blocks * block_threads, dtype=np.uint32)

    def access(self, block, tid, epoch, unit, action, space=SHARED):
        self.rows.append((unit, len(self.rows), block, tid, epoch, action, space))
        return self

    def set_counts(self, count, block=None, tid=None):
        if block is None:
            self.counts[:] = count
        elif tid is None:
            self.counts[block * self.bt:(block + 1) * self.bt] = count
        else:
            self.counts[block * self.bt + tid] = count
        return self

    def trace(self, max_barriers=None) -> Trace:
        if self.rows:
            cols = list(zip(*self.rows))
            ev = pack(*cols)
        else:
            ev = np.zeros((0, 4), dtype=np.uint32)
        mb = int(self.counts.max()) if max_barriers is None and self.counts.size else (max_barriers or 0)
        return Trace(ev, self.counts.copy(), self.nb, self.bt, self.su, self.gu, mb)


# --- parametric model kernels (inputs of the evolutionary search) -----------------
#
# Each model stands for a small CUDA kernel with grid and block dimensions and
# integer arguments; a trace is what simulating one launch records (Algorithm 3's
# schedule: block, epoch, slot, thread; visit order = serial position).
#
# copy2d (kaldi's _copy_from_mat, Sec. 2): 2-D blocks; thread (x, y) of block
#   (bx, by) has column X = bx * block_x + x and row Y = by * block_y + y; it reads
#   src[Y * a1 + X] and writes dst[Y * a0 + X] (global memory, no barrier). src is
#   units [0, 2^19), dst units [2^19, 2^20), indices taken mod 2^19.
# stencil: 1-D blocks of block_x threads (block_y = 1); thread t writes shared
#   sh[(t * a1) mod 4096], passes one barrier, reads sh[(t * a1 + a0) mod 4096] and
#   writes global out[(block * block_x + t) mod 2^20].
# Arguments are integers (negative ones count as 0).
MODEL_COPY2D, MODEL_STENCIL = 0, 1
MODEL_GLOBAL_UNITS = 1 << 20
MODEL_SHARED_UNITS = 4096
_HALF = 1 << 19


def model_events(model: int, grid: tuple, block: tuple) -> int:
    """Records of one launch of a model kernel."""
    threads = grid[0] * grid[1] * block[0] * block[1]
    return threads * (2 if model == MODEL_COPY2D else 3)


def model_trace(model: int, grid: tuple, block: tuple, args: tuple) -> Trace:
    """Host reference of a model kernel's trace (plain loops over the schedule)."""
    gx, gy = grid
    bxd, byd = block
    a0, a1 = max(0, int(args[0])), max(0, int(args[1]))   # negative arguments count as 0
    nb, bt = gx * gy, bxd * byd
    rows = []
    if model == MODEL_COPY2D:
        for b in range(nb):
            bx, by = b % gx, b // gx
            for slot in range(2):
                for t in range(bt):
                    x, y = t % bxd, t // bxd
                    X, Y = bx * bxd + x, by * byd + y
                    if slot == 0:
                        rows.append(((Y * a1 + X) % _HALF, b, t, 0, READ, GLOBAL))
                    else:
                        rows.append((_HALF + (Y * a0 + X) % _HALF, b, t, 0, WRITE, GLOBAL))
        counts = np.zeros(nb * bt, dtype=np.uint32)
        maxb = 0
    else:
        for b in range(nb):
            for t in range(bt):
                rows.append(((t * a1) % MODEL_SHARED_UNITS, b, t, 0, WRITE, SHARED))
            for slot in range(2):
                for t in range(bt):
                    if slot == 0:
                        rows.append(((t * a1 + a0) % MODEL_SHARED_UNITS, b, t, 1, READ, SHARED))
                    else:
                        rows.append(((b * bxd + t) % MODEL_GLOBAL_UNITS, b, t, 1, WRITE, GLOBAL))
        counts = np.ones(nb * bt, dtype=np.uint32)
        maxb = 1
    if rows:
        unit, blk, tid, ep, act, sp = (np.array(c, dtype=np.int64) for c in zip(*rows))
        ev = pack(unit, np.arange(len(rows)), blk, tid, ep, act, sp)
    else:
        ev = np.zeros((0, 4), dtype=np.uint32)
    return Trace(ev, counts, nb, bt, MODEL_SHARED_UNITS, MODEL_GLOBAL_UNITS, maxb,
                 meta=dict(kind="model", model=model, grid=(gx, gy), block=(bxd, byd), args=(a0, a1)))


def with_statements(tr: Trace, seed: int = DEFAULT_SEED, diverge_p: float = 0.05) -> Trace:
    """The same records with statement words: the statement of a record is its position among its
    thread's accesses of its epoch (threads of a warp run the same program point in lockstep), plus
    64 * epoch; every record of a (block, warp, epoch) that diverges (probability diverge_p, hashed
    from the seed) carries DIVERGED."""
    ev = tr.events
    n = ev.shape[0]
    epoch = (ev[:, 3] >> 16) & 0xFFF
    gt = ev[:, 2].astype(np.int64) * tr.block_threads + (ev[:, 3] & 0xFFFF)
    key = gt * 4096 + epoch
    order = np.argsort(key, kind="stable")
    sk = key[order]
    start = np.ones(n, dtype=bool)
    start[1:] = sk[1:] != sk[:-1]
    grp = np.cumsum(start) - 1
    first = np.flatnonzero(start)
    slot = np.empty(n, dtype=np.int64)
    slot[order] = np.arange(n) - first[grp]
    stmt = (epoch.astype(np.int64) * 64 + np.minimum(slot, 63)).astype(np.uint32)
    warp = ev[:, 2].astype(np.uint64) * 64 + ((ev[:, 3] & 0xFFFF) >> 5).astype(np.uint64)
    h = (np.uint64(seed) ^ (warp * np.uint64(0x9E3779B97F4A7C15)) ^ (epoch.astype(np.uint64) << np.uint64(40)))
    h ^= h >> np.uint64(31)
    h *= np.uint64(0xBF58476D1CE4E5B9)
    h ^= h >> np.uint64(29)
    div = (h % np.uint64(1 << 20)).astype(np.float64) / float(1 << 20) < diverge_p
    stmt = stmt | np.where(div, np.uint32(DIVERGED), np.uint32(0))
    out = dataclasses.replace(tr, flags=tr.flags | WARP_AWARE, stmt=stmt.astype(np.uint32),
                              meta=dict(tr.meta, statements=True, diverge_p=diverge_p))
    return out
