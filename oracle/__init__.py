"""CPU oracle for the memory-model synchronization check.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke entry point and the
benchmark's CPU-baseline leg are the only users. The product (CUDA) path never
imports this package and shares no code with it.

What it computes (arXiv 1905.01833, Sec. 3.2 "Memory-based Synchronization Bug
Detection", Theorem 1, Algorithms 4 and 5; the numbered readings R1..R13 are
this library's readings of the places where the paper is silent):

* Records. Each access record carries (unit, visit_order, block, tid, epoch,
  action, space). ``epoch`` is the number of barriers the thread has passed
  (the paper's per-unit visit order, Sec. 3.2.1 and Algorithm 4); the record's
  ``visit_order`` is the serial position of the access in the simulated
  schedule (Algorithm 3's round robin) and only orders accesses (R3, R4).
* Validation. A barrier count above ``max_barriers`` is bad (kind 1, first
  thread index). A record is bad when block >= n_blocks, tid >= block_threads,
  action == 3, the reserved bit is set, the unit is out of its space's range,
  its epoch exceeds its thread's barrier count, or (unless the UNSORTED flag is
  set) its visit order does not exceed the previous record's (kind 0, first
  record index). Counts are checked before records.
* Conflict (Theorem 1 without its warp refinements, R1; atomics R2; same
  thread and read/read never conflict, R11): two records of one unit conflict
  when their owners differ, at least one writes or is atomic, and they are not
  both atomic. Class WW (0) when both modify, RW (1) when exactly one reads.
* Scopes. Intra-block: same space, block, epoch and unit; owners are global
  thread ids (gtid = block * block_threads + tid). Inter-block (global memory
  only, R7): same unit, different blocks, any epochs; owners are blocks.
* Races (R9, R10). Per group and class, the conflicting pair whose later access
  is earliest in schedule order, with the earliest partner; schedule order is
  (visit_order, record index). Records are emitted in canonical order
  (space, scope, block, epoch, unit, class); inter-block records have
  block = epoch = 0xFFFFFFFF and so follow the intra-block global records.
* Redundant barriers (Algorithm 5, R5, R6, R12). Barrier k of block b separates
  epochs k and k+1 and exists for k < max over the block's threads of the
  barrier count. It is redundant unless some unit of block b (either space) has
  a record of epoch k and one of epoch k+1 that conflict (owners: threads).
  Barriers are judged one at a time. Listed sorted by (block, k). The grid list
  holds each k that is redundant in every block that has barrier k.
* Divergence (Algorithm 4, Sec. 2, R8). A block whose threads' barrier counts
  differ, reported as (block, min, max, lowest tid holding the min), by block.

Pinned by: exhaustive pair checks on tiny traces (tests/bruteforce.py), the
hand-built closed-form cases in tests/, and the paper's worked examples kept
under tests/golden/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simulee_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib_handle = None

OK, EBADTRACE, ENOMEM = 0, 2, 3

RACE_DTYPE = np.dtype([("space", "u1"), ("scope", "u1"), ("cls", "u1"), ("pad", "u1"),
                       ("block", "<u4"), ("epoch", "<u4"), ("unit", "<u4"),
                       ("vo_first", "<u4"), ("vo_second", "<u4"),
                       ("gtid_first", "<u4"), ("gtid_second", "<u4")])
DIV_DTYPE = np.dtype([("block", "<u4"), ("min_count", "<u4"), ("max_count", "<u4"), ("first_min_tid", "<u4")])
BAR_DTYPE = np.dtype([("block", "<u4"), ("barrier", "<u4")])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no GPU)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.orc_check.restype = vp
    lib.orc_check.argtypes = [vp, u64, vp, u32, u32, u32, u32, u32, u32]
    if hasattr(lib, "orc_check2"):
        lib.orc_check2.restype = vp
        lib.orc_check2.argtypes = [vp, u64, vp, u32, u32, u32, u32, u32, u32, vp]
    for name, rt in [("orc_status", ctypes.c_int32), ("orc_bad_kind", u32), ("orc_bad_index", u64),
                     ("orc_n_races", u64), ("orc_n_divs", u64), ("orc_n_bars", u64), ("orc_n_grid", u64)]:
        getattr(lib, name).restype = rt
        getattr(lib, name).argtypes = [vp]
    lib.orc_copy.restype = None
    lib.orc_copy.argtypes = [vp, vp, vp, vp, vp]
    lib.orc_free.restype = None
    lib.orc_free.argtypes = [vp]
    if hasattr(lib, "orc_fitness"):
        lib.orc_fitness.restype = ctypes.c_int32
        lib.orc_fitness.argtypes = [vp, u64, vp, u32, u32, u32, u32, u32, u32, vp, vp, vp, vp, vp]
    return lib


def _lib():
    global _lib_handle
    with _lock:
        if _lib_handle is None:
            _lib_handle = _bind(ctypes.CDLL(build()))
    return _lib_handle


def load(path: str):
    """Bind another build of the oracle source (used by the mutation tests)."""
    return _bind(ctypes.CDLL(path))


WARP_AWARE = 2     # trace flag: records carry statement words (Theorem 1's warp refinements apply)
PAPER_ORDER = 4    # trace flag: the paper's visit-order counters (Algorithm 3) group the tuples
DIVERGED = 0x80000000


def check_arrays(events, barrier_counts, n_blocks, block_threads, shared_units, global_units,
                 max_barriers, flags=0, lib=None, stmt=None) -> dict:
    """Run the oracle on raw arrays; returns status, bad_kind, bad_index and the four lists.
    stmt (with flag WARP_AWARE): per record, statement id | DIVERGED."""
    lib = lib or _lib()
    ev = np.ascontiguousarray(events, dtype=np.uint32).reshape(-1, 4)
    cn = np.ascontiguousarray(barrier_counts, dtype=np.uint32)
    if cn.size != n_blocks * block_threads:
        raise ValueError("barrier_counts must hold n_blocks * block_threads entries")
    if flags & WARP_AWARE:
        st = np.ascontiguousarray(stmt, dtype=np.uint32)
        if st.size != ev.shape[0]:
            raise ValueError("a warp-aware trace needs one statement word per record")
        h = lib.orc_check2(ev.ctypes.data_as(ctypes.c_void_p), ev.shape[0], cn.ctypes.data_as(ctypes.c_void_p),
                           n_blocks, block_threads, shared_units, global_units, max_barriers, flags,
                           st.ctypes.data_as(ctypes.c_void_p))
    else:
        h = lib.orc_check(ev.ctypes.data_as(ctypes.c_void_p), ev.shape[0], cn.ctypes.data_as(ctypes.c_void_p),
                          n_blocks, block_threads, shared_units, global_units, max_barriers, flags)
    if not h:
        raise MemoryError("oracle ran out of host memory")
    try:
        out = dict(status=int(lib.orc_status(h)), bad_kind=int(lib.orc_bad_kind(h)),
                   bad_index=int(lib.orc_bad_index(h)))
        races = np.zeros(lib.orc_n_races(h), dtype=RACE_DTYPE)
        divs = np.zeros(lib.orc_n_divs(h), dtype=DIV_DTYPE)
        bars = np.zeros(lib.orc_n_bars(h), dtype=BAR_DTYPE)
        grid = np.zeros(lib.orc_n_grid(h), dtype=np.uint32)
        lib.orc_copy(h, races.ctypes.data_as(ctypes.c_void_p), divs.ctypes.data_as(ctypes.c_void_p),
                     bars.ctypes.data_as(ctypes.c_void_p), grid.ctypes.data_as(ctypes.c_void_p))
        out.update(races=races, divergence=divs, redundant=bars, grid_redundant=grid)
        return out
    finally:
        lib.orc_free(h)


def check(trace, lib=None) -> dict:
    """Run the oracle on any object with the trace attributes (events, barrier_counts, dims, flags)."""
    return check_arrays(trace.events, trace.barrier_counts, trace.n_blocks, trace.block_threads,
                        trace.shared_units, trace.global_units, trace.max_barriers, getattr(trace, "flags", 0),
                        lib=lib, stmt=getattr(trace, "stmt", None))


def fitness_arrays(events, barrier_counts, n_blocks, block_threads, shared_units, global_units,
                   max_barriers, flags=0, lib=None) -> dict:
    """Eq. 1 of the paper on raw arrays: sum g (addresses accessed), sum f (distinct (address, thread)
    pairs) and the accessed unit range of each space; validation as for check()."""
    lib = lib or _lib()
    ev = np.ascontiguousarray(events, dtype=np.uint32).reshape(-1, 4)
    cn = np.ascontiguousarray(barrier_counts, dtype=np.uint32)
    if cn.size != n_blocks * block_threads:
        raise ValueError("barrier_counts must hold n_blocks * block_threads entries")
    kind, idx = ctypes.c_uint32(), ctypes.c_uint64()
    na, npairs = ctypes.c_uint64(), ctypes.c_uint64()
    rng = (ctypes.c_uint32 * 4)()
    st = lib.orc_fitness(ev.ctypes.data_as(ctypes.c_void_p), ev.shape[0], cn.ctypes.data_as(ctypes.c_void_p),
                         n_blocks, block_threads, shared_units, global_units, max_barriers, flags,
                         ctypes.byref(kind), ctypes.byref(idx), ctypes.byref(na), ctypes.byref(npairs), rng)
    if st == ENOMEM:
        raise MemoryError("oracle ran out of host memory")
    return dict(status=int(st), bad_kind=int(kind.value), bad_index=int(idx.value), n_addresses=int(na.value),
                n_pairs=int(npairs.value), shared_lo=int(rng[0]), shared_hi=int(rng[1]), global_lo=int(rng[2]),
                global_hi=int(rng[3]))


def fitness(trace, lib=None) -> dict:
    """fitness_arrays() on a trace object."""
    return fitness_arrays(trace.events, trace.barrier_counts, trace.n_blocks, trace.block_threads,
                          trace.shared_units, trace.global_units, trace.max_barriers, getattr(trace, "flags", 0),
                          lib=lib)
