"""Serving: continuous batching of check jobs on one GPU under an HBM budget.

Jobs (device-resident traces) arrive over time. The loop admits arrived jobs
while their working memory (batch workspace and output buffers) fits in the
budget, launches everything admitted since the last launch as one batched
check (simulee_check_batch) on a free CUDA stream, and keeps up to
`max_inflight` batches running at once, so work that arrives while the GPU is
busy overlaps with the batches already on the device. A finished batch returns
its memory to the budget and its per-job results and latencies (arrival to
results on the host). `serial=True` checks one job at a time, in arrival
order, on one stream: the comparison point.

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


@dataclasses.dataclass
class Job:
    jid: int
    trace: simulee.DeviceTrace
    arrival: float                 # seconds after the start of the run
    races_cap: int = 0
    admitted: float = -1.0
    done: float = -1.0
    result: dict | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _caps(dt: simulee.DeviceTrace, races_cap: int):
    return (races_cap or 2 * dt.n_events + 2, dt.n_blocks, dt.n_blocks * max(dt.max_barriers, 1),
            max(dt.max_barriers, 1))


class _Batch:
    """One launched batched check: its stream, buffers, jobs and completion event."""

    def __init__(self, server, jobs, stream):
        torch = server.torch
        self.jobs = jobs
        self.stream = stream
        T = len(jobs)
        dev = server.dev
        caps = [_caps(j.trace, j.races_cap) for j in jobs]
        widths = (32, 16, 8, 4)
        self.caps = caps
        self.offs = []
        total = [0, 0, 0, 0]
        for c in caps:
            o = []
            for k in range(4):
                o.append(total[k])
                total[k] += c[k] * widths[k]
            self.offs.append(o)
        self.bufs = [torch.empty(max(t, 16), dtype=torch.uint8, device=dev) for t in total]
        outs = (simulee.Outputs * T)()
        for i, c in enumerate(caps):
            o = self.offs[i]
            outs[i] = simulee.Outputs(self.bufs[0].data_ptr() + o[0], c[0], self.bufs[1].data_ptr() + o[1], c[1],
                                      self.bufs[2].data_ptr() + o[2], c[2], self.bufs[3].data_ptr() + o[3], c[3])
        self.reports = torch.zeros(T * simulee.REPORT_BYTES, dtype=torch.uint8, device=dev)
        arr = (simulee.Trace * T)(*[j.trace.c() for j in jobs])
        n = ctypes.c_size_t()
        simulee._check(simulee.lib().simulee_batch_workspace_size(server.chk.h, arr, T, ctypes.byref(n)),
                       "simulee_batch_workspace_size")
        try:
            self.ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
        except torch.OutOfMemoryError:   # cached blocks of finished batches: hand them back, then retry once
            torch.cuda.empty_cache()
            self.ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=dev)
        self.bytes = self.ws.numel() + sum(b.numel() for b in self.bufs) + self.reports.numel()
        with torch.cuda.stream(stream):
            simulee._check(simulee.lib().simulee_check_batch(
                server.chk.h, arr, T, outs, ctypes.c_void_p(self.reports.data_ptr()),
                ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), ctypes.c_void_p(stream.cuda_stream)),
                "simulee_check_batch")
            self.h_reports = torch.empty_like(self.reports, device="cpu").pin_memory()
            self.h_reports.copy_(self.reports, non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(stream)

    def done(self) -> bool:
        return self.event.query()

    def collect(self, keep_lists: bool):
        rep_bytes = self.h_reports.numpy().tobytes()
        host = [b.cpu().numpy() for b in self.bufs] if keep_lists else None
        dts = (simulee.RACE_DTYPE, simulee.DIV_DTYPE, simulee.BAR_DTYPE, np.dtype("<u4"))
        for i, j in enumerate(self.jobs):
            r = simulee.Report.from_buffer_copy(rep_bytes[i * simulee.REPORT_BYTES:(i + 1) * simulee.REPORT_BYTES])
            res = dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                       n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)
            if keep_lists:
                counts = (r.n_races, r.n_divergence, r.n_redundant, r.n_grid_redundant)
                names = ("races", "divergence", "redundant", "grid_redundant")
                ok = r.status in (simulee.OK, simulee.ETRUNC)
                for k in range(4):
                    cnt = min(self.caps[i][k], counts[k]) if ok else 0
                    o = self.offs[i][k]
                    res[names[k]] = np.frombuffer(host[k][o:o + cnt * dts[k].itemsize].tobytes(), dtype=dts[k])
            j.result = res


class Server:
    """Continuous-batching check server on one GPU."""

    def __init__(self, device: int = 0, hbm_budget: int = 120 << 30, max_inflight: int = 3, max_batch: int = 4096,
                 serial: bool = False, keep_lists: bool = True, races_cap: int = 1 << 20):
        import torch
        self.torch = torch
        self.device = device
        self.dev = f"cuda:{device}"
        self.chk = simulee.Checker(device)
        self.budget = hbm_budget
        self.max_inflight = 1 if serial else max_inflight
        self.max_batch = 1 if serial else max_batch
        self.keep_lists = keep_lists
        self.races_cap = races_cap     # per-job race list capacity unless the job sets its own
        self.streams = [torch.cuda.Stream(device) for _ in range(self.max_inflight)]

    def _need(self, job: Job) -> int:
        """Working memory a job adds to a batch: workspace (worst case per record) and outputs."""
        dt = job.trace
        t = dt.c()
        n = ctypes.c_size_t()
        simulee._check(simulee.lib().simulee_workspace_size(self.chk.h, ctypes.byref(t), ctypes.byref(n)),
                       "simulee_workspace_size")
        c = _caps(dt, job.races_cap)
        return int(n.value) + 32 * c[0] + 16 * c[1] + 8 * c[2] + 4 * c[3]

    def _batch_need(self, batch: list[Job]) -> int:
        """Working memory of a batch as one call: its workspace (the batch's key widths and
        signature table, which can exceed the sum of its jobs' own) and outputs."""
        arr = (simulee.Trace * len(batch))(*[j.trace.c() for j in batch])
        n = ctypes.c_size_t()
        simulee._check(simulee.lib().simulee_batch_workspace_size(self.chk.h, arr, len(batch), ctypes.byref(n)),
                       "simulee_batch_workspace_size")
        out = 0
        for j in batch:
            c = _caps(j.trace, j.races_cap)
            out += 32 * c[0] + 16 * c[1] + 8 * c[2] + 4 * c[3]
        return int(n.value) + out

    def run(self, jobs: list[Job], clock=time.perf_counter) -> dict:
        """Serve jobs at their arrival times (seconds after start); returns latency and throughput figures."""
        torch = self.torch
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            if not j.races_cap:
                j.races_cap = min(self.races_cap, 2 * j.trace.n_events + 2)
        need = {j.jid: self._need(j) for j in jobs}
        for j in jobs:
            if need[j.jid] > self.budget:
                raise ValueError(f"job {j.jid} needs {need[j.jid]} bytes, more than the whole budget")
        pending = collections.deque()
        inflight: list[_Batch] = []
        free_streams = list(self.streams)
        used = 0
        nxt = 0
        n_batches, max_batch_seen, max_inflight_seen, max_used = 0, 0, 0, 0
        torch.cuda.synchronize(self.device)
        t0 = clock()
        while nxt < len(jobs) or pending or inflight:
            now = clock() - t0
            while nxt < len(jobs) and jobs[nxt].arrival <= now:
                pending.append(jobs[nxt])
                nxt += 1
            # retire finished batches: results to the host, memory back to the budget
            still = []
            for b in inflight:
                if b.done():
                    b.collect(self.keep_lists)
                    t_done = clock() - t0
                    for j in b.jobs:
                        j.done = t_done
                    used -= b.reserved
                    free_streams.append(b.stream)
                else:
                    still.append(b)
            inflight = still
            # admit and launch everything that arrived and fits
            if pending and free_streams:
                batch, reserve = [], 0
                while pending and len(batch) < self.max_batch and used + reserve + need[pending[0].jid] <= self.budget:
                    j = pending.popleft()
                    reserve += need[j.jid]
                    batch.append(j)
                if batch:
                    # the batch as one call may need more than its jobs' sum: give jobs back until it fits
                    reserve = self._batch_need(batch)
                    while len(batch) > 1 and used + reserve > self.budget:
                        pending.appendleft(batch.pop())
                        reserve = self._batch_need(batch)
                    if used + reserve > self.budget and inflight:
                        pending.extendleft(reversed(batch))   # wait for memory to come back
                        batch = []
                if batch:
                    t_adm = clock() - t0
                    for j in batch:
                        j.admitted = t_adm
                    b = _Batch(self, batch, free_streams.pop())
                    b.reserved = reserve
                    used += reserve
                    inflight.append(b)
                    n_batches += 1
                    max_batch_seen = max(max_batch_seen, len(batch))
                    max_inflight_seen = max(max_inflight_seen, len(inflight))
                    max_used = max(max_used, used)
                    continue
            if not inflight and nxt < len(jobs) and not pending:
                # idle until the next arrival
                wait = jobs[nxt].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
            else:
                time.sleep(2e-5)
        wall = clock() - t0
        lat = np.array([j.latency for j in jobs])
        events = sum(j.trace.n_events for j in jobs)
        return dict(jobs=len(jobs), events=events, wall_s=wall, events_per_s=events / wall,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    max_ms=float(lat.max() * 1e3), mean_ms=float(lat.mean() * 1e3), batches=n_batches,
                    max_batch=max_batch_seen, max_inflight=max_inflight_seen, max_reserved_bytes=max_used)


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """n arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
