"""Benchmark of the synchronization check: access records checked per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Default workload (the headline line): one step = one batched check
(simulee_check_batch: races, divergence and redundant barriers of every trace)
of the batched workload: 4096 independent traces with lognormal sizes (median
1e5 records, clipped to 1e3..1e7, sigma fitted so that the sizes sum to 6e8
records), block sizes {64, 128, 256, 1024}, 4..64 barrier epochs, tree-reduction
and tiled-transpose blocks over shared and global memory (9.6 GB of records,
larger than L2, so no flush is needed between steps).

`value` is measured with the traces resident in HBM; `e2e` times the same
batched check through the C ABI with the traces in pinned host memory,
including the host-to-device copy of every record and the device-to-host copy
of the reports and result lists. `parity` compares every trace's result with
the CPU oracle (rank 0, one GPU), which is also the timed `cpu_baseline`
(one oracle process per host core). The line also carries the plain
single-trace form (`single_trace`: one check of the grid workload, 1024 blocks
x 256 threads, 32 epochs, ~6.1e7 records) and the served form (`served`:
Poisson arrivals of jobs of log-uniform size 1e4..1e8 records under a 120 GB
budget, batched serving against serial checking).

With N > 1 (torchrun) every rank checks its own batch (independent replicas;
the check has no cross-GPU exchange) and the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "access-events checked/sec"
UNIT = "Gev/s"
WORKLOAD = ("grid: 1024 blocks x 256 threads, 32 epochs, 12288 shared units/block + 2^26 global units, "
            "tree-reduction / 32x32 tiled-transpose blocks, 10% blocks missing one barrier, 2% global atomics")
BATCH_WORKLOAD = ("batch: {T} traces, lognormal sizes (median 1e5 records, sigma {sigma:.4f} fitted to a "
                  "{total:.2g}-record total, clipped 1e3..1e7), block sizes 64/128/256/1024, 4..64 epochs, "
                  "tree-reduction / tiled-transpose blocks; one batched check per step")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_min_mhz": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch, dev: int) -> str | None:
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else f"GPU-{s}"
    except Exception:
        return None


def bits(count):
    b = 0
    while (1 << b) < count:
        b += 1
    return b


def sig_slots(tr):
    """Entries of the block-signature table that every check clears (one trace: one per global unit)."""
    if tr.global_units == 0:
        return 0
    if tr.global_units <= (1 << 28):
        return tr.global_units
    m = 1 << 16
    while m < tr.n_events and m < (1 << 28):
        m <<= 1
    return m


def global_counts(tr) -> tuple[int, int]:
    """Global records of the trace, and the global units they touch (each unit's block signature is read and
    written once)."""
    ev = tr.events.reshape(-1, 4)
    g = ev[((ev[:, 3] >> 30) & 1) == 1, 0]
    return int(g.size), (int(np.unique(g).size) if g.size else 0)


def stage_bytes(tr, sizes, path: str, n_gl: int, n_gunits: int):
    """Algorithmic DRAM bytes of each stage for the plan that ran (stream sizes from the library).

    Per record: one 16-byte read. Per global record: the inter-block stream
    element it produces (key + 8-byte payload). Per touched global unit: one
    read and one write of its 4-byte block signature; the signature table is
    cleared once per check. Per routed intra-block element (sort path): its
    key + 8-byte payload written, then read and written by every radix pass,
    then read by the reduction, plus the 16-byte re-read of its record by the
    fallback read (hash path only).
    ingest: count statistics, the signature clear and, on the sort path, the
    first read with all routing. hash: the single read of the hash path.
    fallback: the re-read and routing of what the hash path spilled. sort: the
    inter-block filter and the radix passes. reduce: one read of every sorted
    stream."""
    n = tr.n_events
    n_s, n_g, n_x, n_xs = sizes["n_s"], sizes["n_g"], sizes["n_x"], sizes["x_slots"]
    bb, bus, bug, be = bits(tr.n_blocks), bits(tr.shared_units), bits(tr.global_units), bits(tr.max_barriers + 1)
    ks = 8 if bb + bus + be > 32 else 4
    kg = 8 if bb + bug + be > 32 else 4
    kx = 8 if bug > 32 else 4
    np_s, np_g, np_x = -(-(bb + bus + be) // 8), -(-(bb + bug + be) // 8), -(-bug // 8)
    first = 16 * n + n_gl * (kx + 8) + 8 * n_gunits
    routed = n_s * (ks + 8) + n_g * (kg + 8)
    hashed = path != "sort"
    return dict(
        ingest=4 * tr.barrier_counts.size + 4 * sig_slots(tr) + (0 if hashed else first + routed),
        hash=first if hashed else 0,
        fallback=(16 * (n_s + n_g) + routed) if hashed else 0,
        sort=n_xs * (kx + 8) + n_x * (kx + 8)
        + 2 * (n_s * np_s * (ks + 8) + n_g * np_g * (kg + 8) + n_x * np_x * (kx + 8)),
        reduce=n_s * (ks + 8) + n_g * (kg + 8) + n_x * (kx + 8),
        launches=dict(ingest=1, hash=1, fallback=1, sort=np_s + np_g + np_x + 1, reduce=3))


def kernel_traffic(kernel: str, workload: str):
    """ncu DRAM bytes per launch recorded under profiles/, if the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[f"{kernel}|{workload}"]
    except Exception:
        return None
    src = os.path.join(ROOT, rec["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return rec["bytes_per_launch"] if h == rec["source_sha"] else None


def run_oracle_sample(tr, n_blocks: int):
    """Time the CPU oracle on the records of the first n_blocks blocks (a bounded sample)."""
    import oracle
    import tracegen
    sel = tr.events[:, 2] < n_blocks
    st = getattr(tr, "stmt", None)
    sub = tracegen.Trace(tr.events[sel].copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units,
                         tr.global_units, tr.max_barriers, tr.flags, stmt=None if st is None else st[sel].copy())
    t0 = time.perf_counter()
    out = oracle.check(sub)
    dt = time.perf_counter() - t0
    assert out["status"] == 0
    return int(sel.sum()), dt


def make_trace(rank: int, n_blocks: int = 1024):
    import tracegen
    return tracegen.c2(seed=tracegen.DEFAULT_SEED + rank, n_blocks=n_blocks)


def job_value(events_this_rank: int, ms_this_rank: float, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: all ranks' records over the slowest rank's time.

    Returns (Gev/s, max ms). With torch.distributed initialised (NCCL on the GPU machine, gloo in the
    CPU tests) the time is the max over ranks and the records are summed over ranks."""
    ms, total = float(ms_this_rank), float(events_this_rank)
    if dist is not None and dist.is_initialized():
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        n = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        ms, total = float(t.item()), float(n.item())
    return total / (ms * 1e-3) / 1e9, ms


def device_pool(torch, trs, dev):
    """Upload many host traces into one device buffer; DeviceTrace views into it."""
    from paper_1905_01833_gb300 import simulee
    n = sum(t.n_events for t in trs)
    m = sum(t.barrier_counts.size for t in trs)
    ev = torch.empty((max(n, 1), 4), dtype=torch.int32, device=dev)
    cn = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    out, a, b = [], 0, 0
    for t in trs:
        k, c = t.n_events, t.barrier_counts.size
        if k:
            ev[a:a + k].copy_(torch.from_numpy(t.events.view(np.int32)))
        cn[b:b + c].copy_(torch.from_numpy(t.barrier_counts.view(np.int32)))
        out.append(simulee.DeviceTrace(ev[a:a + k], cn[b:b + c], t.n_blocks, t.block_threads, t.shared_units,
                                       t.global_units, t.max_barriers, t.flags))
        a += k
        b += c
    return out, (ev, cn)


def result_digest(res: dict, races_cap: int) -> str:
    """Digest of one trace's result: status, counts and the list bytes (the race list up to races_cap,
    the length an output of that capacity holds). An oracle result and a GPU result with that race
    capacity have equal digests exactly when they are identical."""
    nr = int(res["n_races"]) if "n_races" in res else len(res["races"])
    status = int(res["status"])
    if status == 4 and nr > races_cap:   # truncated race list: the prefix and the true count are compared
        status = 0
    h = hashlib.sha256()
    h.update(np.array([status, int(res["bad_kind"]), int(res["bad_index"]), nr, len(res["divergence"]),
                       len(res["redundant"]), len(res["grid_redundant"])], dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(res["races"][:races_cap]).tobytes())
    for k in ("divergence", "redundant", "grid_redundant"):
        h.update(np.ascontiguousarray(res[k]).tobytes())
    return h.hexdigest()


def batch_specs(seed: int, n_traces: int):
    """Member specs (index, records, block size, epochs, seed) of the batched workload, and its sigma
    (fitted to 6e8 records for 4096 traces, in proportion for other counts)."""
    import tracegen
    total = tracegen.C3_RECORDS * n_traces // 4096
    sigma = tracegen.c3_sigma(seed=seed, n_traces=n_traces, total=total)
    sizes, bss, eps = tracegen.c3_sizes(seed=seed, n_traces=n_traces, sigma=sigma)
    return [(i, int(n), int(b), int(e), seed) for i, (n, b, e) in enumerate(zip(sizes, bss, eps))], sigma


def race_cap_for(n: int) -> int:
    """Race-list capacity of a batch member in the parity call (its true count fits with room to spare)."""
    return min(2 * n + 2, 1024 + n // 8)


# ---- the oracle on the host cores: one spawned process per core ----------------------------------

def _oracle_host(conn, barrier):
    """One oracle process: builds batch members on request, then checks them with the oracle, timed
    from a common start (a barrier shared by all processes) to its last member."""
    import oracle
    import tracegen
    cache = {}
    while True:
        msg = conn.recv()
        if msg[0] == "quit":
            break
        if msg[0] == "gen":
            for spec in msg[1]:
                i, n, bs, ep, seed = spec
                cache[i] = tracegen.c3_trace(i, n, bs, ep, seed=seed)
            conn.send(len(cache))
        elif msg[0] == "run":
            ids, want_digest = msg[1], msg[2]
            barrier.wait()
            t0 = time.monotonic()
            res = []
            for i in ids:
                res.append(oracle.check(cache[i]))
            t1 = time.monotonic()
            out = []
            for i, r in zip(ids, res):
                assert r["status"] == 0, f"oracle status {r['status']} on member {i}"
                out.append((i, cache[i].n_events, result_digest(r, race_cap_for(cache[i].n_events))
                            if want_digest else None))
            conn.send((t0, t1, out))
        elif msg[0] == "drop":
            cache.clear()
            conn.send(0)


class OracleHosts:
    """The CPU oracle in one spawned process per host core (spawned before any GPU work)."""

    def __init__(self, cores: int | None = None):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = cores or len(os.sched_getaffinity(0))
        self.barrier = ctx.Barrier(self.cores)
        self.conns, self.procs = [], []
        for _ in range(self.cores):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_host, args=(b, self.barrier), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        self.assign: list[list[int]] = [[] for _ in range(self.cores)]

    def generate(self, specs):
        """Spread members over the processes by records (longest first) and have them build the traces."""
        loads = [0] * self.cores
        parts = [[] for _ in range(self.cores)]
        for spec in sorted(specs, key=lambda s: -s[1]):
            w = loads.index(min(loads))
            parts[w].append(spec)
            loads[w] += spec[1]
        for c, p in zip(self.conns, parts):
            c.send(("gen", p))
        for c in self.conns:
            c.recv()
        self.assign = [[s[0] for s in p] for p in parts]

    def run(self, want_digest: bool):
        """Check every member once; returns (wall seconds from common start to last finish, records,
        {member: digest})."""
        for c, ids in zip(self.conns, self.assign):
            c.send(("run", ids, want_digest))
        outs = [c.recv() for c in self.conns]
        t0 = min(o[0] for o in outs)
        t1 = max(o[1] for o in outs)
        n, dig = 0, {}
        for o in outs:
            for i, k, d in o[2]:
                n += k
                dig[i] = d
        return t1 - t0, n, dig

    def close(self):
        for c in self.conns:
            try:
                c.send(("quit",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)


# ---- batched workload on the GPU ----------------------------------------------------------------

def generate_members(specs, threads: int):
    import tracegen
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda s: tracegen.c3_trace(s[0], s[1], s[2], s[3], seed=s[4]), specs))


def member_global_counts(trs, threads: int):
    """Per member: global records and distinct global units (the hash path's inter-block stream and
    signature bytes)."""
    def one(tr):
        ev = tr.events
        g = ev[((ev[:, 3] >> 30) & 1) == 1, 0]
        return int(g.size), (int(np.unique(g).size) if g.size else 0)
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, trs))


def batch_key_bytes(trs) -> int:
    """Bytes of an inter-block stream key in a batched call over these traces (8 when wider than 32 bits)."""
    return 8 if bits(len(trs)) + bits(max(t.global_units for t in trs)) > 32 else 4


class BatchRun:
    """Buffers and C-ABI calls of one batched check over device-resident traces."""

    def __init__(self, torch, dts, device: str, caps, compact: bool = True, **opts):
        import ctypes
        from paper_1905_01833_gb300 import simulee
        self.torch, self.simulee, self.ctypes = torch, simulee, ctypes
        self.dev = device
        self.chk = simulee.Checker(int(device.split(":")[1]), **opts)
        self.T = len(dts)
        self.arr = (simulee.Trace * self.T)(*[d.c() for d in dts])
        self.set_caps(caps)
        self.reports = torch.zeros(self.T * simulee.REPORT_BYTES, dtype=torch.uint8, device=device)
        self.set_workspace(compact)

    def set_workspace(self, compact: bool):
        """A compact workspace (simulee_compact_workspace_size) or the one that never runs out of room."""
        simulee, ctypes = self.simulee, self.ctypes
        n = ctypes.c_size_t()
        f = simulee.lib().simulee_compact_workspace_size if compact else simulee.lib().simulee_batch_workspace_size
        simulee._check(f(self.chk.h, self.arr, self.T, ctypes.byref(n)), "workspace size")
        self.compact = compact
        self.ws = None
        self.ws = self.torch.empty(int(n.value), dtype=self.torch.uint8, device=self.dev)

    def set_caps(self, caps):
        """Output lists: per member (races, divergence, redundant, grid) capacities, packed per kind."""
        simulee, torch = self.simulee, self.torch
        widths = (32, 16, 8, 4)
        self.caps = caps
        self.offs = []
        tot = [0, 0, 0, 0]
        for c in caps:
            self.offs.append(tuple(tot))
            tot = [tot[k] + c[k] * widths[k] for k in range(4)]
        self.bufs = [torch.empty(max(x, 16), dtype=torch.uint8, device=self.dev) for x in tot]
        self.used = tot
        self.outs = (simulee.Outputs * self.T)()
        for i, c in enumerate(caps):
            o = self.offs[i]
            self.outs[i] = simulee.Outputs(*(v for k in range(4) for v in (self.bufs[k].data_ptr() + o[k], c[k])))

    def call(self, stream, arr=None, chk=None, reports_ptr=None):
        c = self.ctypes
        h = (chk or self.chk).h
        s = self.simulee.lib().simulee_check_batch(h, arr if arr is not None else self.arr, self.T, self.outs,
                                                   c.c_void_p(reports_ptr or self.reports.data_ptr()),
                                                   c.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                                   c.c_void_p(stream.cuda_stream))
        if s != 0:
            raise RuntimeError(f"simulee_check_batch failed: {self.simulee.status_str(s)}")

    def hash_groups(self, stream) -> dict:
        """Blocks per hash-path launch group in the last call on this run's workspace (simulee_hash_groups)."""
        c, torch = self.ctypes, self.torch
        out = torch.zeros(5, dtype=torch.int32, device=self.dev)
        self.simulee._check(self.simulee.lib().simulee_hash_groups(
            self.chk.h, c.c_void_p(self.ws.data_ptr()), c.c_void_p(out.data_ptr()), c.c_void_p(stream.cuda_stream)),
            "simulee_hash_groups")
        v = [int(x) for x in out.cpu().tolist()]
        return dict(zip(("quarter", "half", "small", "large"), (v[i + 1] - v[i] for i in range(4))))

    def stream_sizes(self, stream) -> dict:
        """Stream counts of the last call on this run's workspace (simulee_stream_sizes)."""
        c, torch = self.ctypes, self.torch
        out = torch.zeros(5, dtype=torch.int32, device=self.dev)
        self.simulee._check(self.simulee.lib().simulee_stream_sizes(
            self.chk.h, c.c_void_p(self.ws.data_ptr()), c.c_void_p(out.data_ptr()), c.c_void_p(stream.cuda_stream)),
            "simulee_stream_sizes")
        v = [int(x) for x in out.cpu().tolist()]
        return dict(n_s=v[0], n_g=v[1], n_x=v[2], n_races=v[3], x_slots=v[4])

    def results(self, reports_host=None):
        """Per member: report fields and host copies of its lists."""
        simulee = self.simulee
        rb = (reports_host if reports_host is not None else self.reports.cpu()).numpy().tobytes()
        host = [b.cpu().numpy() for b in self.bufs]
        dts = (simulee.RACE_DTYPE, simulee.DIV_DTYPE, simulee.BAR_DTYPE, np.dtype("<u4"))
        names = ("races", "divergence", "redundant", "grid_redundant")
        out = []
        for i in range(self.T):
            r = simulee.Report.from_buffer_copy(rb[i * simulee.REPORT_BYTES:(i + 1) * simulee.REPORT_BYTES])
            res = dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                       n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)
            counts = (r.n_races, r.n_divergence, r.n_redundant, r.n_grid_redundant)
            ok = r.status in (simulee.OK, simulee.ETRUNC)
            for k in range(4):
                cnt = min(self.caps[i][k], counts[k]) if ok else 0
                o = self.offs[i][k]
                res[names[k]] = np.frombuffer(host[k][o:o + cnt * dts[k].itemsize].tobytes(), dtype=dts[k])
            out.append(res)
        return out


def batch_stage_bytes(trs, gcounts, sizes, kx: int):
    """Algorithmic DRAM bytes of the stages of one batched check (the hash path's plan).

    hash: one 16-byte read of every record, the inter-block stream element (key + 8-byte payload) of
    every global record, a read and a write of the block signature of every touched global unit.
    sort: the inter-block filter (every slot read, every kept element written) and the radix passes of
    the streams the library reports (elements read and written per pass). ingest: barrier counts and
    the signature-table clear. reduce: one read of every sorted stream."""
    n = sum(t.n_events for t in trs)
    n_gl = sum(g for g, _ in gcounts)
    n_gu = sum(u for _, u in gcounts)
    n_s, n_g, n_x, n_xs = sizes["n_s"], sizes["n_g"], sizes["n_x"], sizes["x_slots"]
    T = len(trs)
    bb = bits(sum(t.n_blocks for t in trs))
    bus = bits(max(t.shared_units for t in trs))
    bug = bits(max(t.global_units for t in trs))
    be = bits(max(t.max_barriers for t in trs) + 1)
    ks = 8 if bb + bus + be > 32 else 4
    kg = 8 if bb + bug + be > 32 else 4
    np_s, np_g, np_x = -(-(bb + bus + be) // 8), -(-(bb + bug + be) // 8), -(-(bits(T) + bug) // 8)
    sig = 4 * sum(t.global_units for t in trs)
    return dict(
        ingest=sum(4 * t.barrier_counts.size for t in trs) + sig,
        hash=16 * n + n_gl * (kx + 8) + 8 * n_gu,
        fallback=16 * (n_s + n_g) + n_s * (ks + 8) + n_g * (kg + 8),
        sort=n_xs * (kx + 8) + n_x * (kx + 8)
        + 2 * (n_s * np_s * (ks + 8) + n_g * np_g * (kg + 8) + n_x * np_x * (kx + 8)),
        reduce=n_s * (ks + 8) + n_g * (kg + 8) + n_x * (kx + 8),
        n_records=n, n_global=n_gl, n_global_units=n_gu, radix_passes=np_s + np_g + np_x)


def headline(args, rank: int, world: int, local: int, dist):
    """The batched workload: device time, end to end, roofline of the hash stage, oracle parity and
    baseline; plus the single-trace and served forms on one GPU."""
    import torch
    import tracegen
    from paper_1905_01833_gb300 import simulee
    dev = f"cuda:{local}"
    cores = len(os.sched_getaffinity(0))
    specs, sigma = batch_specs(tracegen.DEFAULT_SEED + rank, args.batch_traces)
    with_oracle = rank == 0 and world == 1 and not args.no_cpu_baseline
    hosts = OracleHosts() if with_oracle else None   # spawned before the first GPU call
    t0 = time.perf_counter()
    trs = generate_members(specs, cores)
    gen_s = time.perf_counter() - t0
    gcounts = member_global_counts(trs, cores)
    oracle_line = None
    if hosts is not None:
        hosts.generate(specs)
        wall, n_or, digests = hosts.run(want_digest=True)
        hosts.close()
        oracle_line = {"value": n_or / wall / 1e9, "unit": UNIT, "cores": hosts.cores, "kind": "oracle",
                       "sample": f"every member of the batch ({len(specs)} traces, {n_or} records), one oracle "
                                 f"process per host core, {wall:.1f} s wall from a common start"}

    torch.cuda.set_device(local)
    dts, keep = device_pool(torch, trs, dev)
    T = len(dts)
    n_ev = sum(d.n_events for d in dts)
    stream = torch.cuda.current_stream()
    # parity call: generous race capacities; its counts size the lists of the timed calls
    # launch choices (radix width and tile, hash-vs-sort cutover, CTA shapes and counts) from the autotuner
    tune_info, tuned = None, {}
    if not args.no_autotune:
        from paper_1905_01833_gb300 import autotune
        t0 = time.perf_counter()
        tuner = autotune.Autotuner(local, cache_path=args.autotune_cache)
        tuned = tuner.best_batch(dts, races_caps=[race_cap_for(d.n_events) for d in dts])
        hit = tuner.cache.get(tuner.batch_key(dts), {})
        tune_info = {"options": tuned, "bucket": tuner.batch_key(dts), "tuned_ms": hit.get("ms"),
                     "default_ms": hit.get("default_ms"), "evaluated": hit.get("evaluated"),
                     "seconds": time.perf_counter() - t0}
    run = BatchRun(torch, dts, dev, [(race_cap_for(d.n_events), d.n_blocks, d.n_blocks * max(d.max_barriers, 1),
                                      max(d.max_barriers, 1)) for d in dts],
                   **dict(tuned, graph_replay=simulee.GRAPH_OFF if args.graph_replay == "off" else simulee.GRAPH_AUTO))
    run.call(stream)
    torch.cuda.synchronize()
    first = run.results()
    if any(r["status"] == simulee.ENOMEM for r in first):   # the compact workspace ran out of room
        run.set_workspace(compact=False)
        run.call(stream)
        torch.cuda.synchronize()
        first = run.results()
    bad = [i for i, r in enumerate(first) if r["status"] != 0]
    if bad:
        raise RuntimeError(f"batch member {bad[0]} reported status {first[bad[0]]['status']}")
    parity = None
    if hosts is not None:
        eq = [i for i in range(T) if result_digest(first[i], race_cap_for(dts[i].n_events)) == digests[i]]
        ne = sorted(set(range(T)) - set(eq))
        parity = {"checked": T, "equal": len(eq), "first_mismatch": ne[0] if ne else None,
                  "what": "every member's status, counts and race / divergence / redundant-barrier / grid lists, "
                          "byte for byte against the CPU oracle"}
    counts = [(r["n_races"], r["n_divergence"], r["n_redundant"], r["n_grid_redundant"]) for r in first]
    run.set_caps([tuple(max(int(x), 1) for x in c) for c in counts])   # exact-size lists for the timed calls
    for _ in range(args.warmup):
        run.call(stream)
    torch.cuda.synchronize()
    launches = run.chk.last_launches()
    sampler = ClockSampler(gpu_uuid(torch, local) if world == 1 else None)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run.call(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    again = run.results()
    for i in range(T):   # the timed calls give the parity call's results
        if again[i]["n_races"] != counts[i][0] or again[i]["status"] != 0:
            raise RuntimeError(f"batch member {i}: timed call differs from the parity call")
    # per-stage times from further calls with the library's stage events (launched directly)
    nst = len(simulee.STAGES)
    reps = 3
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nst)] for _ in range(reps)]
    for row in sev:
        for e in row:
            e.record(stream)
    for row in sev:
        run.chk.set_stage_events(row)
        run.call(stream)
    torch.cuda.synchronize()
    run.chk.set_stage_events(None)
    stage_ms = {name: sum(r[2 * k].elapsed_time(r[2 * k + 1]) for r in sev) / reps
                for k, name in enumerate(simulee.STAGES)}
    n_hash = run.chk.last_launches()
    sizes = run.stream_sizes(stream)
    hgroups = run.hash_groups(stream)
    value, ms = job_value(n_ev, ms, dist, dev)

    # end to end: every step copies all records and counts from pinned host memory, checks the batch
    # and reads the reports and result lists back; two device copies of the batch (the resident one
    # and a second), the next step's upload on a copy stream while this step is checked
    ev_h = torch.empty(keep[0].shape, dtype=torch.int32).pin_memory()
    cn_h = torch.empty(keep[1].shape, dtype=torch.int32).pin_memory()
    ev_h.copy_(keep[0])
    cn_h.copy_(keep[1])
    ev2, cn2 = torch.empty_like(keep[0]), torch.empty_like(keep[1])
    base_e, base_c = keep[0].data_ptr(), keep[1].data_ptr()
    arr2 = (simulee.Trace * T)()
    for i, d in enumerate(dts):
        c = d.c()
        if d.n_events:
            c.events = ev2.data_ptr() + (d.events.data_ptr() - base_e)
        c.barrier_counts = cn2.data_ptr() + (d.barrier_counts.data_ptr() - base_c)
        arr2[i] = c
    arrs = [run.arr, arr2]
    d_ev, d_cn = [keep[0], ev2], [keep[1], cn2]
    chks = [run.chk, simulee.Checker(local, **tuned)]
    copy_s = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    rep_h = torch.empty(T * simulee.REPORT_BYTES, dtype=torch.uint8).pin_memory()
    out_h = [torch.empty(max(u, 16), dtype=torch.uint8).pin_memory() for u in run.used]
    h2d = ev_h.numel() * 4 + cn_h.numel() * 4
    d2h = T * simulee.REPORT_BYTES + sum(run.used)

    def issue_copy(i):
        q = i % 2
        if i >= 2:
            copy_s.wait_event(freed[q])
        with torch.cuda.stream(copy_s):
            d_ev[q].copy_(ev_h, non_blocking=True)
            d_cn[q].copy_(cn_h, non_blocking=True)
        copied[q].record(copy_s)

    def finish_step(i):
        q = i % 2
        stream.wait_event(copied[q])
        run.call(stream, arr=arrs[q], chk=chks[q])
        freed[q].record(stream)
        rep_h.copy_(run.reports, non_blocking=True)
        for k in range(4):
            if run.used[k]:
                out_h[k][:run.used[k]].copy_(run.bufs[k][:run.used[k]], non_blocking=True)
        stream.synchronize()

    def run_e2e(k, overlap):
        issue_copy(0)
        for i in range(k):
            if overlap and i + 1 < k:
                issue_copy(i + 1)
            finish_step(i)
            if not overlap and i + 1 < k:
                issue_copy(i + 1)

    run_e2e(3, True)
    e2e_sampler = ClockSampler(gpu_uuid(torch, local) if world == 1 else None)
    e2e_sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_e2e(args.e2e_steps, True)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_value, _ = job_value(n_ev, e2e_s * 1e3, dist, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nser = max(2, args.e2e_steps // 2)
    run_e2e(nser, False)
    e2e_serial, _ = job_value(n_ev, (time.perf_counter() - t0) / nser * 1e3, dist, dev)
    e2e_clocks = e2e_sampler.stop()
    # the upload alone (device time on the copy stream): the host link's bound on the end-to-end figure
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    u0.record(copy_s)
    for _ in range(3):
        with torch.cuda.stream(copy_s):
            d_ev[1].copy_(ev_h, non_blocking=True)
            d_cn[1].copy_(cn_h, non_blocking=True)
    u1.record(copy_s)
    torch.cuda.synchronize()
    upload_ms = u0.elapsed_time(u1) / 3
    link_value, _ = job_value(n_ev, upload_ms, dist, dev)
    chks[1].close()
    rb = rep_h.numpy().tobytes()
    for i in range(T):
        r = simulee.Report.from_buffer_copy(rb[i * simulee.REPORT_BYTES:(i + 1) * simulee.REPORT_BYTES])
        if r.status != 0 or r.n_races != counts[i][0]:
            raise RuntimeError(f"batch member {i}: end-to-end result differs from the resident-trace check")
    del ev2, cn2, ev_h, cn_h, out_h

    # roofline of the dominant stage (the hash path's single read)
    peak, peak_src = peaks()
    sb = batch_stage_bytes(trs, gcounts, sizes, batch_key_bytes(trs))
    cand = [k for k in ("ingest", "hash", "fallback", "sort", "reduce") if sb[k] > 0]
    dom = max(cand, key=lambda k: stage_ms[k])
    kname = {"ingest": "k_block_stats", "hash": "k_hash_blocks", "fallback": "k_ingest", "sort": "k_onesweep",
             "reduce": "k_reduce_groups"}[dom]
    # the hash kernel runs one launch per launch group that holds blocks (thread groups of 128 or 256
    # threads in the smaller CTAs, whole smaller CTAs, larger CTAs)
    nl = max(1, sum(1 for v in hgroups.values() if v > 0)) if dom == "hash" else 1
    achieved = sb[dom] / (stage_ms[dom] * 1e-3) / 1e9
    b_plan = sum(sb[k] for k in ("ingest", "hash", "fallback", "sort", "reduce")) / n_ev
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "launches": nl, "hash_groups": hgroups,
                "bytes_per_launch": sb[dom] / nl, "launch_ms": stage_ms[dom] / nl,
                "stage_bytes": sb[dom], "stage_ms": stage_ms[dom],
                "bytes_per_record": sb[dom] / n_ev,
                "traffic": kernel_traffic(kname, "batch"),
                "plan": {"bytes_per_record": b_plan, "frac": value * 1e9 * b_plan / (peak * 1e9),
                         "floor_frac": value * 1e9 * 16 / (peak * 1e9), "radix_passes": sb["radix_passes"]}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(T=T, sigma=sigma, total=float(n_ev)), "traces": T,
                   "n_events": n_ev, "sigma": sigma, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (9.6 GB of records, 129 MB L2); no flush",
                   "launch": "repeated identical batched calls replayed by the library as one CUDA graph"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "serial_value": e2e_serial,
                "overlap": "two device copies of the batch: the next step's host-to-device copy runs on a copy "
                           "stream while the current step is checked; serial_value = copy, check and read-back "
                           "one after another",
                "link": {"upload_ms": upload_ms, "h2d_gbs": h2d / (upload_ms * 1e-3) / 1e9, "bound_value": link_value,
                         "what": "the step's upload alone from pinned host memory (CUDA events on the copy "
                                 "stream, 3 copies); bound_value = records per second that link carries, the "
                                 "ceiling of value when the check overlaps the upload"},
                "clocks": e2e_clocks},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "stages_ms": stage_ms,
        "streams": sizes,
        "workspace_bytes": run.ws.numel(),
        "workspace_bytes_per_record": run.ws.numel() / n_ev,
        "workspace": "compact" if run.compact else "full",
        "generation_s": gen_s,
        "results": {"n_races": int(sum(c[0] for c in counts)), "n_divergence": int(sum(c[1] for c in counts)),
                    "n_redundant": int(sum(c[2] for c in counts)), "n_grid_redundant": int(sum(c[3] for c in counts))},
        "clocks": clocks,
    }
    if tune_info:
        line["autotune"] = tune_info
    if oracle_line:
        line["cpu_baseline"] = oracle_line
    if parity:
        line["parity"] = parity
    del run, dts, keep, trs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


def reference_arm(args, rank: int, world: int):
    """The oracle as the reference arm: each step checks a bounded sample of the batched workload (every
    ref_stride-th member) with one oracle process per host core; rank 0 only."""
    if rank != 0:
        return
    import tracegen
    specs, sigma = batch_specs(tracegen.DEFAULT_SEED, args.batch_traces)
    sample = specs[::args.ref_stride]
    hosts = OracleHosts(min(len(os.sched_getaffinity(0)), len(sample)))
    hosts.generate(sample)
    for _ in range(args.warmup):
        hosts.run(want_digest=False)
    times, n = [], 0
    for _ in range(args.steps):
        wall, n, _ = hosts.run(want_digest=False)
        times.append(wall)
    hosts.close()
    t = sum(times) / len(times)
    v = n / t / 1e9
    total = sum(s[1] for s in specs)
    desc = (f"every {args.ref_stride}th member of the batched workload ({len(sample)} traces, {n} records) per "
            f"step, one oracle process per host core ({hosts.cores})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(T=len(specs), sigma=sigma, total=float(total)),
                   "traces": len(specs), "n_events": total, "sigma": sigma, "n_events_per_step": n},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": hosts.cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def single_trace_arm(args):
    """One more single-trace configuration: 'strided' (1 block x 256 threads, 8 epochs, 32768 records) or
    'barrier' (1024 blocks x 1024 threads, 64 epochs, 2^28 records). Device time of simulee_check with the
    trace resident, and the oracle on a sample."""
    import torch
    import tracegen
    from paper_1905_01833_gb300 import simulee
    if args.workload == "strided":
        tr, name, sample_blocks = tracegen.c1(), "strided: 1 block x 256 threads, 8 epochs, 12288 shared units", 1
    elif args.workload == "warp":
        tr = tracegen.with_statements(make_trace(0, args.blocks), diverge_p=0.05)
        name = ("warp-aware (Theorem 1 with its warp conditions): the grid workload with a statement word per "
                "record, 5% of (block, warp, epoch) diverged; radix-sort path, pairwise group search")
        sample_blocks = 16
    elif args.workload == "paper":
        tr = make_trace(0, args.blocks)
        tr.flags |= tracegen.PAPER_ORDER
        name = ("paper visit orders (Algorithm 3's counters): the grid workload with flag PAPER_ORDER; radix-sort "
                "path, visit orders of global records by a segmented scan, inter-block groups per visit order")
        sample_blocks = 16
    else:
        tr, name = tracegen.c4(), "barrier: 1024 blocks x 1024 threads, 64 epochs, 4 accesses per thread per epoch"
        sample_blocks = 8
    dt = simulee.to_device(tr)
    # launch choices (radix width and tile, hash-vs-sort cutover, CTA shapes and counts) from the autotuner
    opts = {}
    if not args.no_autotune:
        from paper_1905_01833_gb300 import autotune
        opts = autotune.Autotuner(0, cache_path=args.autotune_cache).best(dt)
    chk = simulee.Checker(0, **opts)
    races_cap = min(2 * tr.n_events + 2, 1 << 22)
    ws = chk.workspace(chk.workspace_size(dt))
    outs, bufs = chk.alloc_outputs(races_cap, tr.n_blocks, tr.n_blocks * max(tr.max_barriers, 1),
                                   max(tr.max_barriers, 1))
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda:0")
    t = dt.c()
    stream = torch.cuda.current_stream()
    import ctypes
    L = simulee.lib()

    def step():
        st = L.simulee_check(chk.h, ctypes.byref(t), ctypes.byref(outs), ctypes.c_void_p(rep.data_ptr()),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(stream.cuda_stream))
        if st != simulee.OK:
            raise RuntimeError(simulee.status_str(st))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 50 if args.workload == "barrier" else 500))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    r = simulee.Report.from_buffer_copy(rep.cpu().numpy().tobytes())
    line = {"workload": name, "n_events": tr.n_events, "value": tr.n_events / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "launches_per_step": chk.last_launches(),
            "options": opts or "library defaults",
            "results": {"status": r.status, "n_races": r.n_races, "n_divergence": r.n_divergence,
                        "n_redundant": r.n_redundant, "n_grid_redundant": r.n_grid_redundant}}
    if not args.no_cpu_baseline:
        n, secs = run_oracle_sample(tr, sample_blocks)
        line["cpu_baseline"] = {"value": n / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"records of blocks 0..{sample_blocks - 1} ({n} records, {secs:.2f} s)"}
    return line


def fitness_arm(args):
    """Fitness of Eq. 1 (distinct addresses / distinct address-thread pairs) over the grid workload: records
    per second through simulee_fitness_batch, with the plan's algorithmic bytes against the HBM peak."""
    import ctypes
    import torch
    import tracegen
    from paper_1905_01833_gb300 import simulee
    tr = make_trace(0, args.blocks)
    dt = simulee.to_device(tr)
    chk = simulee.Checker(0)
    arr = (simulee.Trace * 1)(dt.c())
    ws = chk.workspace(chk.fitness_workspace_size([dt]))
    out = torch.zeros(simulee.FITNESS_BYTES, dtype=torch.uint8, device="cuda:0")
    stream = torch.cuda.current_stream()
    L = simulee.lib()

    def step():
        st = L.simulee_fitness_batch(chk.h, arr, 1, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel(), ctypes.c_void_p(stream.cuda_stream))
        if st != simulee.OK:
            raise RuntimeError(f"simulee_fitness_batch failed: {simulee.status_str(st)}")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = chk.last_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 50))
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    f = simulee.Fitness.from_buffer_copy(out.cpu().numpy().tobytes())
    assert f.status == 0
    # key bits of the radix sort that takes what the single read leaves (here: nothing; every block's
    # distinct pairs fit its table): gtid + unit + block + space
    kb = bits(tr.n_blocks * tr.block_threads) + bits(max(tr.shared_units, tr.global_units)) + bits(tr.n_blocks) + 1
    npass = -(-kb // 8)
    n = tr.n_events
    # HBM bytes: the validation read and the single read of every record, the barrier counts; the block
    # tables (512 KB per CTA) and the global-unit bitmap stay in L2
    algo = n * (16 + 16) + 4 * tr.barrier_counts.size
    peak, peak_src = peaks()
    line = {"workload": f"fitness (Eq. 1) over the grid workload ({tr.n_blocks} blocks, {n} records)",
            "unit": UNIT, "value": n / (ms * 1e-3) / 1e9, "ms_per_step": ms, "steps": steps,
            "launches_per_step": launches, "key_bits": kb, "radix_passes": npass,
            "result": {"n_addresses": f.n_addresses, "n_pairs": f.n_pairs, "F": f.n_addresses / max(f.n_pairs, 1),
                       "shared_range": [f.shared_lo, f.shared_hi], "global_range": [f.global_lo, f.global_hi]},
            "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": algo / (ms * 1e-3) / 1e9 / peak, "peak_source": peak_src,
                         "bytes_per_step": algo}}
    if not args.no_cpu_baseline:
        import oracle
        sel = tr.events[:, 2] < args.oracle_blocks
        sub = tracegen.Trace(tr.events[sel].copy(), tr.barrier_counts, tr.n_blocks, tr.block_threads,
                             tr.shared_units, tr.global_units, tr.max_barriers)
        t0 = time.perf_counter()
        o = oracle.fitness(sub)
        secs = time.perf_counter() - t0
        assert o["status"] == 0
        line["cpu_baseline"] = {"value": int(sel.sum()) / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"records of blocks 0..{args.oracle_blocks - 1} ({int(sel.sum())} records, "
                                          f"{secs:.1f} s, single thread)"}
    return line


def evolve_arm(args):
    """Evolutionary search (Algorithms 1 and 2: population 50, 3 generations, acceptable F < 0.3) over the
    copy2d and stencil model kernels at full dimension limits: every generation's children are generated on
    the device and scored by one batched fitness call; the best launch is then checked."""
    import torch
    from paper_1905_01833_gb300 import evolve, simulee
    chk = simulee.Checker(0)
    scorer = evolve.DeviceScorer(chk)
    out = {"workload": "evolve: population 50, 3 generations, copy2d (grid <= 16x16, block <= 32x32) and stencil "
                       "(grid <= 64, block <= 1024)", "unit": "candidates/s", "models": {}}
    for name, model in (("copy2d", simulee.MODEL_COPY2D), ("stencil", simulee.MODEL_STENCIL)):
        ev = evolve.Evolution(model, scorer, population=50, generations=3, seed=args.steps)
        calls = {"n": 0, "records": 0, "secs": 0.0}

        def timed(sols, _inner=scorer):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = _inner(sols)
            torch.cuda.synchronize()
            calls["secs"] += time.perf_counter() - t0
            calls["n"] += len(sols)
            calls["records"] += sum(tracegen_events(s) for s in sols)
            return res
        ev.scorer = timed
        timed([ev.initial() for _ in range(4)])   # warm-up
        calls.update(n=0, records=0, secs=0.0)
        t0 = time.perf_counter()
        r = ev.run()
        wall = time.perf_counter() - t0
        rep = evolve.detect(chk, r["best"])
        b = r["best"]
        out["models"][name] = {
            "candidates": calls["n"], "records": calls["records"], "scoring_s": calls["secs"], "wall_s": wall,
            "value": calls["n"] / calls["secs"], "records_per_s": calls["records"] / calls["secs"],
            "generations": r["generations"], "accepted": r["accepted"], "best_F": b.F, "best_R": b.R,
            "best_launch": {"grid": b.dims[:2], "block": b.dims[2:], "args": [int(a) for a in b.args]},
            "check": {"status": rep["status"], "races": len(rep["races"]), "redundant": len(rep["redundant"]),
                      "divergence": len(rep["divergence"])}}
    return out


def tracegen_events(sol) -> int:
    import tracegen
    model, grid, block, _ = sol.launch()
    return tracegen.model_events(model, grid, block)


def grid_arm(args, rank: int, world: int, local: int, dist, full: bool = True):
    """The plain single-trace form: one simulee_check of the grid workload per step, trace resident in HBM;
    with `full`, also direct launches, end to end through the C ABI and the oracle on a sample."""
    import ctypes
    import torch
    from paper_1905_01833_gb300 import simulee
    torch.cuda.set_device(local)
    tr = make_trace(rank, args.blocks)
    dt = simulee.to_device(tr, f"cuda:{local}")
    mode = dict(path=simulee.PATH_SORT if args.path == "sort" else simulee.PATH_AUTO, hash_shape=args.hash_shape,
                graph_replay=simulee.GRAPH_OFF if args.graph_replay == "off" else simulee.GRAPH_AUTO)
    chk = simulee.Checker(local, **mode)
    ws = chk.workspace(chk.compact_workspace_size([dt]))
    compact = True
    caps = dict(races_cap=4_000_000, div_cap=tr.n_blocks, red_cap=tr.n_blocks * tr.max_barriers,
                grid_cap=tr.max_barriers)
    outs, bufs = chk.alloc_outputs(caps["races_cap"], caps["div_cap"], caps["red_cap"], caps["grid_cap"])
    report_dev = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    L = simulee.lib()
    ctrace = dt.c()
    sp = ctypes.c_void_p(stream.cuda_stream)

    def step(c, trace_c, rep_ptr):
        s = L.simulee_check(c.h, ctypes.byref(trace_c), ctypes.byref(outs), ctypes.c_void_p(rep_ptr),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), sp)
        if s != 0:
            raise RuntimeError(f"simulee_check failed: {simulee.status_str(s)}")

    step(chk, ctrace, report_dev.data_ptr())
    torch.cuda.synchronize()
    if simulee.Report.from_buffer_copy(report_dev.cpu().numpy().tobytes()).status == simulee.ENOMEM:
        ws = None
        ws = chk.workspace(chk.workspace_size(dt))   # the compact workspace ran out of room
        compact = False
    for _ in range(args.warmup):
        step(chk, ctrace, report_dev.data_ptr())
    torch.cuda.synchronize()
    rep0 = simulee.Report.from_buffer_copy(report_dev.cpu().numpy().tobytes())
    if rep0.status != 0:
        raise RuntimeError(f"check reported status {rep0.status}")
    launches = chk.last_launches()
    nst = len(simulee.STAGES)
    steps = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nst)] for _ in range(steps)]
    for row in evs:
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid(torch, local) if (world == 1 and full) else None)
    if full:
        sampler.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(steps):
        step(chk, ctrace, report_dev.data_ptr())
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if full else None
    ms = t_start.elapsed_time(t_end) / steps
    for i in range(steps):
        chk.set_stage_events(evs[i])
        step(chk, ctrace, report_dev.data_ptr())
    torch.cuda.synchronize()
    chk.set_stage_events(None)
    stage_ms = {name: sum(evs[i][2 * s].elapsed_time(evs[i][2 * s + 1]) for i in range(steps)) / steps
                for s, name in enumerate(simulee.STAGES)}
    rep = simulee.Report.from_buffer_copy(report_dev.cpu().numpy().tobytes())
    assert rep.status == 0 and rep.n_races == rep0.n_races and rep.n_redundant == rep0.n_redundant
    direct = None
    if world == 1:
        chk_d = simulee.Checker(local, **dict(mode, graph_replay=simulee.GRAPH_OFF))
        for _ in range(3):
            step(chk_d, ctrace, report_dev.data_ptr())
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(steps):
            step(chk_d, ctrace, report_dev.data_ptr())
        g1.record(stream)
        torch.cuda.synchronize()
        ms_d = g0.elapsed_time(g1) / steps
        direct = {"value": tr.n_events / (ms_d * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_d,
                  "launches_per_step": chk_d.last_launches()}
        chk_d.close()
    value, ms = job_value(tr.n_events, ms, dist, f"cuda:{local}")

    sizes = chk.stream_sizes()
    hgroups = chk.hash_groups()
    sb = stage_bytes(tr, sizes, args.path, *global_counts(tr))
    sb["launches"]["hash"] = max(1, sum(1 for v in hgroups.values() if v > 0))
    peak, peak_src = peaks()
    cand = [k for k in ("ingest", "hash", "fallback", "sort", "reduce") if sb[k] > 0]
    dom = max(cand, key=lambda k: stage_ms[k])
    kname = {"ingest": "k_ingest", "hash": "k_hash_blocks", "fallback": "k_ingest", "sort": "k_onesweep",
             "reduce": "k_reduce_groups"}[dom]
    nl = sb["launches"][dom]
    achieved = sb[dom] / (stage_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "bytes_per_launch": sb[dom] / nl, "launch_ms": stage_ms[dom] / nl, "launches": nl,
                "hash_groups": hgroups, "traffic": kernel_traffic(kname, "grid")}
    b_plan = sum(sb[k] for k in ("ingest", "hash", "fallback", "sort", "reduce")) / tr.n_events
    roofline["plan"] = {"bytes_per_record": b_plan, "frac": value * 1e9 * b_plan / (peak * 1e9),
                        "floor_frac": value * 1e9 * 16 / (peak * 1e9), "radix_passes": sb["launches"]["sort"] - 1}
    line = {"workload": WORKLOAD if args.blocks == 1024 else WORKLOAD.replace("1024 blocks", f"{args.blocks} blocks"),
            "n_events": tr.n_events, "value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "launches_per_step": launches, "direct": direct, "roofline": roofline, "stages_ms": stage_ms,
            "streams": sizes, "workspace_bytes": ws.numel(), "workspace_bytes_per_record": ws.numel() / tr.n_events,
            "workspace": "compact" if compact else "full",
            "results": {"n_races": rep.n_races, "n_divergence": rep.n_divergence, "n_redundant": rep.n_redundant,
                        "n_grid_redundant": rep.n_grid_redundant}}
    if not full:
        return line
    line["clocks"] = clocks

    # end to end through the C ABI: pinned host trace -> device, check, report and lists -> host, every
    # step; two device trace buffers and two contexts, the next step's upload on a copy stream
    h_ev = torch.from_numpy(tr.events.view(np.int32)).pin_memory()
    h_cn = torch.from_numpy(tr.barrier_counts.view(np.int32)).pin_memory()
    d_ev = [torch.empty_like(dt.events) for _ in range(2)]
    d_cn = [torch.empty_like(dt.barrier_counts) for _ in range(2)]
    etr = [simulee.DeviceTrace(d_ev[q], d_cn[q], tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units,
                               tr.max_barriers).c() for q in range(2)]
    chks = [chk, simulee.Checker(local, **mode)]
    copy_s = torch.cuda.Stream(device=f"cuda:{local}")
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    rep_host = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8).pin_memory()
    h_races = torch.empty(caps["races_cap"] * 32, dtype=torch.uint8).pin_memory()
    h_red = torch.empty(max(caps["red_cap"], 1) * 8, dtype=torch.uint8).pin_memory()
    h_div = torch.empty(max(caps["div_cap"], 1) * 16, dtype=torch.uint8).pin_memory()
    h_grid = torch.empty(max(caps["grid_cap"], 1) * 4, dtype=torch.uint8).pin_memory()
    d2h = 0

    def issue_copy(i):
        q = i % 2
        if i >= 2:
            copy_s.wait_event(freed[q])
        with torch.cuda.stream(copy_s):
            d_ev[q].copy_(h_ev, non_blocking=True)
            d_cn[q].copy_(h_cn, non_blocking=True)
        copied[q].record(copy_s)

    def finish_step(i):
        nonlocal d2h
        q = i % 2
        stream.wait_event(copied[q])
        step(chks[q], etr[q], rep_host.data_ptr())
        freed[q].record(stream)
        stream.synchronize()
        r = simulee.Report.from_buffer_copy(rep_host.numpy().tobytes())
        nr, nd, nred, ng = (min(r.n_races, caps["races_cap"]), min(r.n_divergence, caps["div_cap"]),
                            min(r.n_redundant, caps["red_cap"]), min(r.n_grid_redundant, caps["grid_cap"]))
        h_races[: nr * 32].copy_(bufs["races"][: nr * 32], non_blocking=True)
        h_div[: nd * 16].copy_(bufs["divergence"][: nd * 16], non_blocking=True)
        h_red[: nred * 8].copy_(bufs["redundant"][: nred * 8], non_blocking=True)
        h_grid[: ng * 4].copy_(bufs["grid"][: ng * 4], non_blocking=True)
        stream.synchronize()
        d2h = simulee.REPORT_BYTES + nr * 32 + nd * 16 + nred * 8 + ng * 4
        if r.status != 0 or r.n_races != rep0.n_races:
            raise RuntimeError("end-to-end check result differs from the resident-trace check")

    def run_e2e(k, overlap):
        issue_copy(0)
        for i in range(k):
            if overlap and i + 1 < k:
                issue_copy(i + 1)
            finish_step(i)
            if not overlap and i + 1 < k:
                issue_copy(i + 1)

    run_e2e(4, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_e2e(args.e2e_steps, True)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nser = max(2, args.e2e_steps // 2)
    run_e2e(nser, False)
    e2e_serial_s = (time.perf_counter() - t0) / nser
    chks[1].close()
    line["e2e"] = {"value": tr.n_events / e2e_s / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": tr.events.nbytes + tr.barrier_counts.nbytes, "d2h_bytes_per_step": d2h,
                   "serial_value": tr.n_events / e2e_serial_s / 1e9}
    line["gpu_launches"] = launches * steps
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, secs = run_oracle_sample(tr, args.oracle_blocks)
        line["cpu_baseline"] = {"value": n / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"records of blocks 0..{args.oracle_blocks - 1} of the same trace "
                                          f"({n} records, {secs:.1f} s, single thread)",
                                "host_cores": len(os.sched_getaffinity(0))}
    del d_ev, d_cn, dt, ws
    torch.cuda.empty_cache()
    return line


def serve_pool(torch, n_pool: int, dev: str):
    """The served workload's device-resident traces (tracegen.c5_member: sizes log-spaced over 1e4..1e8
    records, grid and barrier families), with each trace's plan bytes on the hash path (record read,
    inter-block elements, signatures)."""
    import tracegen
    pool_sizes = tracegen.c5_pool_sizes(n_pool)
    trs = [tracegen.c5_member(i, sz) for i, sz in enumerate(pool_sizes)]
    plan = []
    for tr in trs:
        g, u = global_counts(tr)
        kx = 8 if bits(tr.global_units) > 32 else 4
        plan.append(16 * tr.n_events + g * (kx + 8) + 8 * u)
    dts, keep = device_pool(torch, trs, dev)
    return trs, dts, keep, pool_sizes, plan


def serve_arm(args):
    """Served workload: Poisson arrivals of check jobs (sizes log-uniform 1e4..1e8 records, picked from a
    pool of device-resident grid- and barrier-family traces), continuous batching under a 120 GB HBM
    budget, against serial checking; at 200 jobs/s and at a rate beyond saturation."""
    import torch
    from paper_1905_01833_gb300 import serve
    trs, dts, keep, pool_sizes, plan = serve_pool(torch, args.serve_pool, "cuda:0")
    rng = np.random.default_rng(7)
    draws = np.exp(rng.uniform(np.log(1e4), np.log(1e8), size=args.serve_jobs))
    pick = np.abs(np.log(draws)[:, None] - np.log(pool_sizes)[None, :]).argmin(axis=1)
    peak, _ = peaks()

    opts = {}
    if not args.no_autotune:
        from paper_1905_01833_gb300 import autotune
        opts = autotune.Autotuner(0, cache_path=args.autotune_cache).best_batch(dts)

    def run(rate, serial):
        arr = serve.poisson_arrivals(rate, args.serve_jobs, seed=11)
        jobs = [serve.Job(i, dts[int(pick[i])], float(arr[i])) for i in range(args.serve_jobs)]
        srv = serve.Server(0, hbm_budget=120 << 30, serial=serial, keep_lists=False, options=opts)
        out = srv.run(jobs)
        b = sum(plan[int(pick[i])] for i in range(args.serve_jobs))
        out["plan_bytes_per_record"] = b / out["events"]
        out["plan_frac"] = b / out["wall_s"] / (peak * 1e9)
        del srv
        torch.cuda.empty_cache()
        return out

    warm = serve.Server(0, keep_lists=False)
    warm.run([serve.Job(i, dts[i % len(dts)], 0.0) for i in range(len(dts))])
    del warm
    torch.cuda.empty_cache()
    keys = ("p50_ms", "p99_ms", "max_ms", "batches", "max_batch", "max_inflight", "plan_frac",
            "plan_bytes_per_record", "jobs", "events", "wall_s")
    res = {"workload": f"serve: Poisson arrivals, {args.serve_jobs} jobs, sizes log-uniform 1e4..1e8 records "
                       f"(pool of {len(dts)} device-resident grid / barrier traces), 120 GB budget, up to 3 "
                       f"batches in flight", "unit": UNIT, "options": opts, "rates": {}}
    for rate in args.serve_rates:
        a = run(rate, serial=False)
        b = run(rate, serial=True)
        res["rates"][str(int(rate))] = {
            "batched": {k: a[k] for k in keys} | {"value": a["events_per_s"] / 1e9},
            "serial": {k: b[k] for k in keys} | {"value": b["events_per_s"] / 1e9}}
    del dts, keep
    torch.cuda.empty_cache()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", choices=["auto", "sort"], default="auto")
    ap.add_argument("--hash-shape", type=int, choices=[0, 1, 2], default=0,
                    help="hash path CTAs: 0 chosen per call, 1 one 1024-thread CTA per SM, 2 two 512-thread CTAs")
    ap.add_argument("--graph-replay", choices=["auto", "off"], default="auto",
                    help="auto: repeated identical calls replayed by the library as one CUDA graph; off: direct launches")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--oracle-blocks", type=int, default=256)
    ap.add_argument("--ref-stride", type=int, default=64, help="reference arm: every n-th batch member per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline: the batched line only")
    ap.add_argument("--no-autotune", action="store_true", help="the library's default launch choices (headline and single-trace arms)")
    ap.add_argument("--autotune-cache", default=None, help="autotuner cache file (default: the user's cache)")
    ap.add_argument("--blocks", type=int, default=1024, help="grid blocks (1024 = the single-trace workload; "
                    "smaller values only for profiling captures)")
    ap.add_argument("--workload", choices=["headline", "grid", "serve", "fitness", "evolve", "strided", "barrier",
                                           "warp", "paper"], default="headline",
                    help="headline: the batched workload with the single-trace and served forms; the others print "
                         "their own line")
    ap.add_argument("--batch-traces", type=int, default=4096)
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 20000.0])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload not in ("headline", "grid"):
        import torch
        torch.cuda.set_device(0)
        out = {"serve": serve_arm, "fitness": fitness_arm, "evolve": evolve_arm, "strided": single_trace_arm,
               "barrier": single_trace_arm, "warp": single_trace_arm, "paper": single_trace_arm}[args.workload](args)
        print(json.dumps({"metric": METRIC, **out}))
        return

    import torch
    dist = None
    if world > 1:
        torch.cuda.set_device(local)
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    if args.workload == "grid":
        line = grid_arm(args, rank, world, local, dist)
        out = {"metric": METRIC, "value": line.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": line.pop("ms_per_step"), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
               "config": {"workload": line.pop("workload"), "n_events": line.pop("n_events"),
                          "parallelism": f"replicas{world}", "path": args.path,
                          "l2": "inputs larger than L2 (1 GB trace, 129 MB L2); no flush"}, **line}
        if rank == 0:
            print(json.dumps(out))
    else:
        line = headline(args, rank, world, local, dist)
        if world == 1 and not args.no_extras:
            line["single_trace"] = grid_arm(args, rank, world, local, None)
            line["served"] = serve_arm(args)
        if rank == 0:
            print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
