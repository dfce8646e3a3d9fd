"""Autotuner for the check's launch choices, with a persistent JSON cache.

Tuned per GPU model and shape bucket (single traces: log2 of the record count,
the block count and the epoch count, and the trace flags; batches: log2 of the trace count and of the
record count, and the share of records in blocks of at most 256 threads). The
knobs are launch-time choices of the library (simulee_options):

* path: the hash path where it applies, or the radix-sort path for everything;
* hash_shape: the hash path's CTAs (one 768-thread CTA per SM with 8192-entry
  run tables, two 512-thread CTAs with 4096-entry tables, or chosen per call);
* hash_cap_eighths / hash_pool_div: the cutover from the hash path to the sort
  path: how full a run's table may get in distinct units (4/8 to 7/8) and how
  many racy units a run resolves in place (table / 3 down to table / 64);
* hash_groups: whether the smaller CTAs check blocks with short runs in thread
  groups of 128 or 256 threads (four or two blocks per CTA at once) or each
  block with the whole CTA;
* hot_unit_marks: whether a warp marks a global unit's block signature once
  per run of lanes holding it (a guard against units every thread reads) or
  once per record (a little less work when no unit is that hot);
* sort_items: the radix sort's tile (256 threads x 8 or 16 elements);
* radix_bits: the radix sort's digit width (6, 8 or 11 bits);
* ingest_ctas_per_sm, sort_ctas_per_sm, reduce_ctas_per_sm: persistent CTAs per
  SM of the record reads, the radix passes and the segmented reductions.

A search is coordinate descent from the library's defaults: each knob in turn
takes the value with the lowest median time of a few calls (CUDA events on the
caller's stream), the others held at the best so far, for two sweeps. Option
sets whose calls report an error (a compact workspace running out of room) are
skipped. The fastest set is cached and reused for inputs of the same bucket.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import statistics

from . import simulee

KNOBS = {
    "path": (simulee.PATH_AUTO, simulee.PATH_SORT),
    "hash_shape": (0, 1, 2),
    "hash_cap_eighths": (7, 6, 5),
    "hash_pool_div": (3, 6, 12),
    "hot_unit_marks": (0, 2),
    "hash_groups": (0, 1),
    "sort_items": (16, 8),
    "radix_bits": (8, 6, 11),
    "ingest_ctas_per_sm": (2, 1),
    "sort_ctas_per_sm": (3, 2),
    "reduce_ctas_per_sm": (3, 2, 4),
}
DEFAULTS = {k: v[0] for k, v in KNOBS.items()}
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "simulee_gb300", "autotune.json")


def _lg(x) -> int:
    return int(math.ceil(math.log2(max(int(x), 1))))


def bucket(dt) -> str:
    """Shape bucket of a trace: log2 ceilings of records, blocks and epochs, and the trace flags that change
    the path (unsorted, warp-aware and paper-order traces take the radix sort)."""
    b = f"n{_lg(dt.n_events)}-b{_lg(dt.n_blocks)}-e{_lg(dt.max_barriers + 1)}"
    flags = int(getattr(dt, "flags", 0) or 0)
    return f"{b}-f{flags}" if flags else b


def batch_bucket(dts) -> str:
    """Shape bucket of a batch: log2 ceilings of traces and records, and the share of records in blocks of at
    most 256 threads (quarters)."""
    n = sum(d.n_events for d in dts)
    small = sum(d.n_events for d in dts if d.block_threads <= 256)
    return f"batch-t{_lg(len(dts))}-n{_lg(n)}-s{int(4 * small / max(n, 1))}"


class Autotuner:
    def __init__(self, device: int = 0, cache_path: str | None = None):
        import torch
        self.torch = torch
        self.device = device
        self.gpu = torch.cuda.get_device_name(device)
        self.cache_path = cache_path or DEFAULT_CACHE
        self.cache = self._load()
        self.evaluations = 0

    def _load(self) -> dict:
        try:
            with open(self.cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
        tmp = self.cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def key(self, dt) -> str:
        return f"{self.gpu}|{bucket(dt)}"

    def batch_key(self, dts) -> str:
        return f"{self.gpu}|{batch_bucket(dts)}"

    # ---- timing -------------------------------------------------------------------------------
    def _time_call(self, chk, arr, T, outs, reps, stream_ptr, ws, ws_bytes, rep, batch: bool):
        torch = self.torch
        L = simulee.lib()

        def once():
            if batch:
                s = L.simulee_check_batch(chk.h, arr, T, outs, ctypes.c_void_p(rep.data_ptr()),
                                          ctypes.c_void_p(ws.data_ptr()), ws_bytes, stream_ptr)
            else:
                s = L.simulee_check(chk.h, ctypes.byref(arr), ctypes.byref(outs), ctypes.c_void_p(rep.data_ptr()),
                                    ctypes.c_void_p(ws.data_ptr()), ws_bytes, stream_ptr)
            if s != simulee.OK:
                raise simulee.SimuleeError(s, "check")
        once()
        torch.cuda.synchronize(self.device)
        stat = rep.view(torch.int32)[:: simulee.REPORT_BYTES // 4].cpu()
        if bool(((stat != simulee.OK) & (stat != simulee.ETRUNC)).any()):
            return math.inf   # e.g. a compact workspace that ran out of room under these options
        times = []
        stream = torch.cuda.current_stream(self.device)
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            once()
            b.record(stream)
            torch.cuda.synchronize(self.device)
            times.append(a.elapsed_time(b))
        return statistics.median(times)

    def time_options(self, dt, opts: dict, reps: int = 3) -> float:
        """Median milliseconds of one full check of a single trace with the given options."""
        torch = self.torch
        chk = simulee.Checker(self.device, **opts)
        try:
            ws_bytes = chk.compact_workspace_size([dt])
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device=f"cuda:{self.device}")
            outs, _ = chk.alloc_outputs(min(2 * dt.n_events + 2, 1 << 20), dt.n_blocks,
                                        dt.n_blocks * max(dt.max_barriers, 1), max(dt.max_barriers, 1))
            rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device=f"cuda:{self.device}")
            sp = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
            self.evaluations += 1
            return self._time_call(chk, dt.c(), 1, outs, reps, sp, ws, ws_bytes, rep, batch=False)
        finally:
            chk.close()

    def time_batch_options(self, dts, opts: dict, reps: int = 3, races_caps=None) -> float:
        """Median milliseconds of one batched check of these traces with the given options."""
        torch = self.torch
        chk = simulee.Checker(self.device, **opts)
        dev = f"cuda:{self.device}"
        try:
            T = len(dts)
            arr = (simulee.Trace * T)(*[d.c() for d in dts])
            rc = races_caps or [min(2 * d.n_events + 2, 1024 + d.n_events // 8) for d in dts]
            caps = [(rc[i], d.n_blocks, d.n_blocks * max(d.max_barriers, 1), max(d.max_barriers, 1))
                    for i, d in enumerate(dts)]
            widths = (32, 16, 8, 4)
            tot = [sum(c[k] * widths[k] for c in caps) for k in range(4)]
            bufs = [torch.empty(max(x, 16), dtype=torch.uint8, device=dev) for x in tot]
            outs = (simulee.Outputs * T)()
            off = [0, 0, 0, 0]
            for i, c in enumerate(caps):
                outs[i] = simulee.Outputs(*(v for k in range(4) for v in (bufs[k].data_ptr() + off[k], c[k])))
                for k in range(4):
                    off[k] += c[k] * widths[k]
            ws_bytes = chk.compact_workspace_size(dts)
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
            rep = torch.zeros(T * simulee.REPORT_BYTES, dtype=torch.uint8, device=dev)
            sp = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
            self.evaluations += 1
            return self._time_call(chk, arr, T, outs, reps, sp, ws, ws_bytes, rep, batch=True)
        finally:
            chk.close()

    # ---- search -------------------------------------------------------------------------------
    def _descend(self, measure, sweeps: int = 2, knobs=None) -> tuple[dict, float, list]:
        """Coordinate descent over the knobs from the defaults; returns (best, its ms, all evaluations)."""
        best = dict(DEFAULTS)
        best_ms = measure(best)
        log = [(dict(best), best_ms)]
        for _ in range(sweeps):
            changed = False
            for k in (knobs or KNOBS):
                for v in KNOBS[k]:
                    if v == best[k]:
                        continue
                    cand = dict(best, **{k: v})
                    if cand["path"] == simulee.PATH_SORT and (k.startswith("hash") or k == "hot_unit_marks"):
                        continue   # the hash knobs do nothing on the sort path
                    ms = measure(cand)
                    log.append((cand, ms))
                    if ms < best_ms:
                        best, best_ms, changed = cand, ms, True
            if not changed:
                break
        return best, best_ms, log

    def tune(self, dt, reps: int = 3, knobs=None, sweeps: int = 2) -> dict:
        best, ms, _ = self._descend(lambda o: self.time_options(dt, o, reps), sweeps=sweeps, knobs=knobs)
        self.cache[self.key(dt)] = dict(best, ms=ms, n_events=dt.n_events)
        self._save()
        return best

    def tune_batch(self, dts, reps: int = 3, knobs=None, races_caps=None, sweeps: int = 2) -> dict:
        best, ms, log = self._descend(lambda o: self.time_batch_options(dts, o, reps, races_caps), sweeps=sweeps,
                                      knobs=knobs)
        self.cache[self.batch_key(dts)] = dict(best, ms=ms, n_events=sum(d.n_events for d in dts),
                                               default_ms=log[0][1], evaluated=len(log))
        self._save()
        return best

    def _hit(self, key):
        hit = self.cache.get(key)
        if hit and all(k in hit for k in KNOBS):
            return {k: hit[k] for k in KNOBS}
        return None

    def best(self, dt) -> dict:
        """Cached options for this trace's bucket, tuning on a miss."""
        return self._hit(self.key(dt)) or self.tune(dt)

    def best_batch(self, dts, **kw) -> dict:
        """Cached options for this batch's bucket, tuning on a miss."""
        return self._hit(self.batch_key(dts)) or self.tune_batch(dts, **kw)

    def checker(self, dt) -> simulee.Checker:
        return simulee.Checker(self.device, **self.best(dt))
