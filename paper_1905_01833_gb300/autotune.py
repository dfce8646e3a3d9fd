"""Autotuner for the check's launch choices, with a persistent JSON cache.

Tuned per GPU model and trace-shape bucket (log2 of the record count, of the
block count and of the epoch count): the path (hash path where it applies, or
the radix-sort path for everything), the hash path's CTA shape (one 1024-thread
CTA per SM with 8192-entry run tables, or two 512-thread CTAs with 4096-entry
tables), and the persistent CTAs per SM of the record reads, the radix passes
and the segmented reductions. Tile sizes and the 8-bit radix are fixed at
compile time. Each candidate is timed
with CUDA events on the caller's trace; the fastest is cached and reused for
traces in the same bucket.
"""
from __future__ import annotations

import ctypes
import itertools
import json
import math
import os
import statistics

from . import simulee

KNOBS = ("path", "hash_shape", "ingest_ctas_per_sm", "sort_ctas_per_sm", "reduce_ctas_per_sm")
# the hash path's shape only matters on the auto path
CANDIDATES = [dict(zip(KNOBS, v)) for v in itertools.product((simulee.PATH_AUTO,), (1, 2), (1, 2), (2, 3), (2, 3, 4))] + \
             [dict(zip(KNOBS, v)) for v in itertools.product((simulee.PATH_SORT,), (0,), (1, 2), (2, 3), (2, 3, 4))]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "simulee_gb300", "autotune.json")


def bucket(dt) -> str:
    """Shape bucket of a trace: log2 ceilings of records, blocks and epochs."""
    def lg(x):
        return int(math.ceil(math.log2(max(int(x), 1))))
    return f"n{lg(dt.n_events)}-b{lg(dt.n_blocks)}-e{lg(dt.max_barriers + 1)}"


class Autotuner:
    def __init__(self, device: int = 0, cache_path: str | None = None):
        import torch
        self.torch = torch
        self.device = device
        self.gpu = torch.cuda.get_device_name(device)
        self.cache_path = cache_path or DEFAULT_CACHE
        self.cache = self._load()

    def _load(self) -> dict:
        try:
            with open(self.cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def _save(self):
        os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
        tmp = self.cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def key(self, dt) -> str:
        return f"{self.gpu}|{bucket(dt)}"

    def time_options(self, dt, opts: dict, reps: int = 3) -> float:
        """Median milliseconds of one full check with the given options."""
        torch = self.torch
        chk = simulee.Checker(self.device, **opts)
        ws = chk.workspace(chk.workspace_size(dt))
        outs, _ = chk.alloc_outputs(min(2 * dt.n_events + 2, 1 << 20), dt.n_blocks, dt.n_blocks * max(dt.max_barriers, 1),
                                    max(dt.max_barriers, 1))
        rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device=f"cuda:{self.device}")
        t = dt.c()
        stream = torch.cuda.current_stream(self.device)
        L = simulee.lib()

        def once():
            s = L.simulee_check(chk.h, ctypes.byref(t), ctypes.byref(outs), ctypes.c_void_p(rep.data_ptr()),
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(stream.cuda_stream))
            if s != simulee.OK:
                raise simulee.SimuleeError(s, "simulee_check")
        once()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            once()
            b.record(stream)
            torch.cuda.synchronize(self.device)
            times.append(a.elapsed_time(b))
        chk.close()
        return statistics.median(times)

    def tune(self, dt, reps: int = 3, candidates=None) -> dict:
        results = []
        for opts in candidates or CANDIDATES:
            results.append((self.time_options(dt, opts, reps), opts))
        ms, best = min(results, key=lambda r: r[0])
        self.cache[self.key(dt)] = dict(best, ms=ms, n_events=dt.n_events)
        self._save()
        return best

    def best(self, dt) -> dict:
        """Cached options for this trace's bucket, tuning on a miss."""
        hit = self.cache.get(self.key(dt))
        if hit:
            return {k: hit[k] for k in KNOBS}
        return self.tune(dt)

    def checker(self, dt) -> simulee.Checker:
        return simulee.Checker(self.device, **self.best(dt))
