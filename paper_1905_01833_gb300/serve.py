"""Serving: continuous batching of check jobs on one GPU under an HBM budget.

Jobs (device-resident traces) arrive over time. The server reserves the whole
budget once, as one device buffer (the arena), and carves each batch's working
memory (workspace, output lists, reports) out of it; nothing is allocated
while serving. The loop admits arrived jobs while their working memory fits in
the free part of the arena, launches everything admitted since the last
launch as one batched check (simulee_check_batch) on a free CUDA stream, and
keeps up to `max_inflight` batches running at once, so work that arrives while
the GPU is busy overlaps with the batches already on the device. A finished
batch returns its memory to the arena and its per-job results and latencies
(arrival to results on the host). `serial=True` checks one job at a time, in
arrival order, on one stream: the comparison point.

Each job's result is the same as checking its trace alone (the batched check
groups by trace and never mixes traces), which the tests verify.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import time

import numpy as np

from . import simulee

_ALIGN = 256
_WIDTHS = (32, 16, 8, 4)   # bytes per race, divergence, redundant-barrier and grid-list record


def _up(x: int) -> int:
    return (x + _ALIGN - 1) // _ALIGN * _ALIGN


@dataclasses.dataclass
class Job:
    jid: int
    trace: simulee.DeviceTrace
    arrival: float                 # seconds after the start of the run
    races_cap: int = 0
    admitted: float = -1.0
    done: float = -1.0
    result: dict | None = None
    need: int = 0                  # working memory of the job checked alone (set at arrival)
    full: bool = False             # run with the worst-case workspace (a compact one ran out of room)
    retries: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _caps(dt: simulee.DeviceTrace, races_cap: int):
    return (races_cap or 2 * dt.n_events + 2, dt.n_blocks, dt.n_blocks * max(dt.max_barriers, 1),
            max(dt.max_barriers, 1))


def _out_bytes(caps) -> int:
    return sum(_up(max(c * w, 16)) for c, w in zip(caps, _WIDTHS))


class Arena:
    """First-fit allocator over one device buffer reserved up front (256-byte aligned pieces)."""

    def __init__(self, torch, nbytes: int, device: str):
        self.size = _up(nbytes)
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.base = self.buf.data_ptr()
        self.free = [(0, self.size)]   # (offset, length), sorted by offset, coalesced

    def largest(self) -> int:
        return max((n for _, n in self.free), default=0)

    def alloc(self, nbytes: int):
        n = _up(max(nbytes, _ALIGN))
        for i, (o, m) in enumerate(self.free):
            if m >= n:
                if m == n:
                    del self.free[i]
                else:
                    self.free[i] = (o + n, m - n)
                return o
        return None

    def release(self, off: int, nbytes: int):
        n = _up(max(nbytes, _ALIGN))
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, m in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + m)
            else:
                merged.append((o, m))
        self.free = merged


class _Batch:
    """One launched batched check: its stream, arena piece, jobs and completion event."""

    def __init__(self, server, jobs, slot: int, arr, ws_bytes: int, off: int, total: int):
        torch = server.torch
        self.jobs = jobs
        self.slot = slot
        self.stream = server.streams[slot]
        self.off, self.total = off, total
        T = len(jobs)
        base = server.arena.base + off
        self.ws_ptr = base
        p = base + _up(ws_bytes)
        self.reports_ptr = p
        p += _up(T * simulee.REPORT_BYTES)
        caps = [_caps(j.trace, j.races_cap) for j in jobs]
        self.caps = caps
        self.out_ptrs = []
        outs = (simulee.Outputs * T)()
        for i, c in enumerate(caps):
            ptrs = []
            for k in range(4):
                ptrs.append(p)
                p += _up(max(c[k] * _WIDTHS[k], 16))
            self.out_ptrs.append(ptrs)
            outs[i] = simulee.Outputs(ptrs[0], c[0], ptrs[1], c[1], ptrs[2], c[2], ptrs[3], c[3])
        assert p - base <= total
        self.h_reports = server.h_reports[slot]
        if self.h_reports.numel() < T * simulee.REPORT_BYTES:
            self.h_reports = server.h_reports[slot] = torch.empty(
                2 * T * simulee.REPORT_BYTES, dtype=torch.uint8).pin_memory()
        # the check, the report read-back and the completion event all go on this batch's stream
        simulee._check(simulee.lib().simulee_check_batch(
            server.chk.h, arr, T, outs, ctypes.c_void_p(self.reports_ptr), ctypes.c_void_p(self.ws_ptr), ws_bytes,
            ctypes.c_void_p(self.stream.cuda_stream)), "simulee_check_batch")
        server.copy_back(self.h_reports, self.reports_ptr, T * simulee.REPORT_BYTES, self.stream)
        self.event = server.events[slot]
        self.event.record(self.stream)

    def done(self) -> bool:
        return self.event.query()

    def collect(self, server, keep_lists: bool):
        T = len(self.jobs)
        rep_bytes = self.h_reports[: T * simulee.REPORT_BYTES].numpy().tobytes()
        dts = (simulee.RACE_DTYPE, simulee.DIV_DTYPE, simulee.BAR_DTYPE, np.dtype("<u4"))
        names = ("races", "divergence", "redundant", "grid_redundant")
        for i, j in enumerate(self.jobs):
            r = simulee.Report.from_buffer_copy(rep_bytes[i * simulee.REPORT_BYTES:(i + 1) * simulee.REPORT_BYTES])
            res = dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                       n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)
            if keep_lists:
                counts = (r.n_races, r.n_divergence, r.n_redundant, r.n_grid_redundant)
                ok = r.status in (simulee.OK, simulee.ETRUNC)
                for k in range(4):
                    cnt = min(self.caps[i][k], counts[k]) if ok else 0
                    res[names[k]] = np.frombuffer(server.read_back(self.out_ptrs[i][k], cnt * dts[k].itemsize),
                                                  dtype=dts[k])
            j.result = res


class Server:
    """Continuous-batching check server on one GPU."""

    def __init__(self, device: int = 0, hbm_budget: int = 120 << 30, max_inflight: int = 3, max_batch: int = 4096,
                 serial: bool = False, keep_lists: bool = True, races_cap: int = 1 << 20,
                 max_batch_records: int = 1 << 30, compact: bool = True, options: dict | None = None):
        import torch
        self.torch = torch
        self.device = device
        self.dev = f"cuda:{device}"
        self.chk = simulee.Checker(device, **(options or {}))   # launch choices, e.g. from the autotuner
        self.budget = hbm_budget
        self.max_inflight = 1 if serial else max_inflight
        self.max_batch = 1 if serial else max_batch
        self.max_batch_records = max_batch_records   # a batch closes once it holds this many records
        self.keep_lists = keep_lists
        self.compact = compact          # compact workspaces; a batch that runs out of room is checked again
        self.races_cap = races_cap     # per-job race list capacity unless the job sets its own
        self.streams = [torch.cuda.Stream(device) for _ in range(self.max_inflight)]
        self.events = [torch.cuda.Event() for _ in range(self.max_inflight)]
        self.h_reports = [torch.empty(4096 * simulee.REPORT_BYTES, dtype=torch.uint8).pin_memory()
                          for _ in range(self.max_inflight)]
        self.arena = Arena(torch, hbm_budget, self.dev)

    def copy_back(self, host, ptr: int, nbytes: int, stream):
        """Asynchronous copy of nbytes of the arena at device address ptr into the pinned tensor host,
        on `stream`."""
        off = ptr - self.arena.base
        with self.torch.cuda.stream(stream):
            host[:nbytes].copy_(self.arena.buf[off:off + nbytes], non_blocking=True)

    def read_back(self, ptr: int, nbytes: int) -> bytes:
        off = ptr - self.arena.base
        return self.arena.buf[off:off + nbytes].cpu().numpy().tobytes() if nbytes else b""

    def _ws_bytes(self, arr, T: int, full: bool) -> int:
        n = ctypes.c_size_t()
        if full:
            simulee._check(simulee.lib().simulee_batch_workspace_size(self.chk.h, arr, T, ctypes.byref(n)),
                           "simulee_batch_workspace_size")
        else:
            simulee._check(simulee.lib().simulee_compact_workspace_size(self.chk.h, arr, T, ctypes.byref(n)),
                           "simulee_compact_workspace_size")
        return int(n.value)

    def _job_need(self, job: Job) -> int:
        """Working memory of a job checked alone: workspace (compact unless the job needs the full one),
        report and output lists."""
        arr = (simulee.Trace * 1)(job.trace.c())
        ws = self._ws_bytes(arr, 1, job.full or not self.compact)
        return _up(ws) + _up(simulee.REPORT_BYTES) + _out_bytes(_caps(job.trace, job.races_cap))

    def _batch_plan(self, batch: list[Job]):
        """(trace array, workspace bytes, total bytes) of a batch as one call: its workspace (the
        batch's key widths and signature table can exceed the sum of its jobs' own), reports, outputs."""
        arr = (simulee.Trace * len(batch))(*[j.trace.c() for j in batch])
        ws = self._ws_bytes(arr, len(batch), any(j.full for j in batch) or not self.compact)
        total = _up(ws) + _up(len(batch) * simulee.REPORT_BYTES) + sum(
            _out_bytes(_caps(j.trace, j.races_cap)) for j in batch)
        return arr, ws, total

    def run(self, jobs: list[Job], clock=time.perf_counter) -> dict:
        """Serve jobs at their arrival times (seconds after start); returns latency and throughput figures."""
        torch = self.torch
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            if not j.races_cap:
                j.races_cap = min(self.races_cap, 2 * j.trace.n_events + 2)
        pending = collections.deque()
        inflight: list[_Batch] = []
        free_slots = list(range(self.max_inflight))
        nxt = 0
        n_batches, max_batch_seen, max_inflight_seen, max_used, n_retried = 0, 0, 0, 0, 0
        torch.cuda.synchronize(self.device)
        t0 = clock()
        while nxt < len(jobs) or pending or inflight:
            now = clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival <= now:
                j = jobs[nxt]
                j.need = self._job_need(j)
                if j.need > self.arena.size:
                    raise ValueError(f"job {j.jid} needs {j.need} bytes, more than the whole budget")
                pending.append(j)
                nxt += 1
            # retire finished batches: results to the host, memory back to the arena
            still = []
            for b in inflight:
                if b.done():
                    b.collect(self, self.keep_lists)
                    t_done = clock() - t0
                    redo = []
                    for j in b.jobs:
                        if j.result["status"] == simulee.ENOMEM and not j.full:
                            # the compact workspace ran out of room: check again with the full one
                            j.full, j.retries, j.result = True, j.retries + 1, None
                            j.need = self._job_need(j)
                            redo.append(j)
                        else:
                            j.done = t_done
                    pending.extendleft(reversed(redo))
                    n_retried += len(redo)
                    self.arena.release(b.off, b.total)
                    free_slots.append(b.slot)
                else:
                    still.append(b)
            inflight = still
            # admit and launch everything that arrived and fits
            launched = False
            if pending and free_slots:
                room = self.arena.largest()
                batch, reserve, recs = [], 0, 0
                while (pending and len(batch) < self.max_batch and reserve + pending[0].need <= room
                       and (not batch or (recs + pending[0].trace.n_events <= self.max_batch_records
                                          and pending[0].full == batch[0].full))):
                    j = pending.popleft()
                    reserve += j.need
                    recs += j.trace.n_events
                    batch.append(j)
                off = None
                while batch:
                    arr, ws, total = self._batch_plan(batch)
                    off = self.arena.alloc(total)
                    if off is not None:
                        break
                    if len(batch) == 1:
                        break
                    pending.appendleft(batch.pop())   # the batch as one call needs more: give jobs back
                if batch and off is None:
                    pending.extendleft(reversed(batch))   # wait for memory to come back
                    if not inflight:
                        raise RuntimeError("a job does not fit the arena although nothing is in flight")
                    batch = []
                if batch:
                    t_adm = clock() - t0
                    for j in batch:
                        j.admitted = t_adm
                    b = _Batch(self, batch, free_slots.pop(), arr, ws, off, total)
                    inflight.append(b)
                    n_batches += 1
                    max_batch_seen = max(max_batch_seen, len(batch))
                    max_inflight_seen = max(max_inflight_seen, len(inflight))
                    max_used = max(max_used, self.arena.size - sum(m for _, m in self.arena.free))
                    launched = True
            if launched:
                continue
            if not inflight and nxt < len(jobs) and not pending:
                # idle until the next arrival
                wait = jobs[nxt].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
            elif inflight:
                # wait a little for the oldest batch (its event), or for the next arrival
                time.sleep(2e-5)
        wall = clock() - t0
        lat = np.array([j.latency for j in jobs])
        events = sum(j.trace.n_events for j in jobs)
        return dict(jobs=len(jobs), events=events, wall_s=wall, events_per_s=events / wall,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    max_ms=float(lat.max() * 1e3), mean_ms=float(lat.mean() * 1e3), batches=n_batches,
                    max_batch=max_batch_seen, max_inflight=max_inflight_seen, max_reserved_bytes=max_used,
                    retried=n_retried)


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """n arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
