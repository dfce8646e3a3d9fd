"""Benchmark of the synchronization check: access records checked per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full check (all stages: validation and routing, radix sorts,
segmented reductions with epoch adjacency, canonical race list, divergence and
redundant-barrier lists) of one synthetic trace of the grid workload: 1024
blocks x 256 threads, 32 barrier epochs, 12288 shared units per block and 2^26
global units, tree-reduction and tiled-transpose blocks, ~6e7 records (~1 GB,
larger than L2, so no flush is needed between steps).

`value` is measured with the trace resident in HBM; `e2e` times the same check
through the C ABI with the trace in pinned host memory, including the host to
device copy of the trace and the device to host copy of the report and lists.
With N > 1 (torchrun) every rank checks its own trace (independent replicas;
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "access-events checked/sec"
UNIT = "Gev/s"
WORKLOAD = ("grid: 1024 blocks x 256 threads, 32 epochs, 12288 shared units/block + 2^26 global units, "
            "tree-reduction / 32x32 tiled-transpose blocks, 10% blocks missing one barrier, 2% global atomics")


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
                "reasons": sorted(reasons), "samples": len(sm)}


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


def reference_arm(args, rank: int, world: int):
    """The oracle as the reference: each step checks a bounded sample of the workload on the host."""
    if rank != 0:
        return
    tr = make_trace(0)
    nb = args.ref_blocks
    for _ in range(args.warmup):
        run_oracle_sample(tr, nb)
    times, n = [], 0
    for _ in range(args.steps):
        n, dt = run_oracle_sample(tr, nb)
        times.append(dt)
    t = sum(times) / len(times)
    v = n / t / 1e9
    sample = f"records of blocks 0..{nb - 1} of the grid workload ({n} records) per step, single thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_events_per_step": n},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


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


def batch_arm(args):
    """Batched workload: 4096 independent traces (lognormal sizes, median 1e5 records, block sizes
    64..1024, 4..64 epochs) checked by one batched call; direct launches and CUDA-graph replay."""
    import ctypes
    import torch
    import tracegen
    from paper_1905_01833_gb300 import simulee
    dev = "cuda:0"
    sizes, bss, eps = tracegen.c3_sizes(n_traces=args.batch_traces)
    base = None if args.no_cpu_baseline else batch_oracle_baseline(sizes, bss, eps)
    t0 = time.perf_counter()
    trs = [tracegen.c3_trace(i, int(n), int(bs), int(e)) for i, (n, bs, e) in enumerate(zip(sizes, bss, eps))]
    gen_s = time.perf_counter() - t0
    dts, keep = device_pool(torch, trs, dev)
    del trs
    chk = simulee.Checker(0)
    T = len(dts)
    arr = (simulee.Trace * T)(*[d.c() for d in dts])
    caps = [(min(2 * d.n_events + 2, 1 << 16), d.n_blocks, d.n_blocks * max(d.max_barriers, 1), max(d.max_barriers, 1))
            for d in dts]
    widths = (32, 16, 8, 4)
    tot = [sum(c[k] * widths[k] for c in caps) for k in range(4)]
    bufs = [torch.empty(max(x, 16), dtype=torch.uint8, device=dev) for x in tot]
    outs = (simulee.Outputs * T)()
    off = [0, 0, 0, 0]
    for i, c in enumerate(caps):
        outs[i] = simulee.Outputs(*(v for k in range(4) for v in (bufs[k].data_ptr() + off[k], c[k])))
        for k in range(4):
            off[k] += c[k] * widths[k]
    reports = torch.zeros(T * simulee.REPORT_BYTES, dtype=torch.uint8, device=dev)
    n = ctypes.c_size_t()
    simulee._check(simulee.lib().simulee_batch_workspace_size(chk.h, arr, T, ctypes.byref(n)), "batch ws")
    ws = torch.empty(int(n.value), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    L = simulee.lib()

    def call():
        s_ = L.simulee_check_batch(chk.h, arr, T, outs, ctypes.c_void_p(reports.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(stream.cuda_stream))
        if s_ != 0:
            raise RuntimeError(simulee.status_str(s_))

    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    rep = np.frombuffer(reports.cpu().numpy().tobytes(), dtype=np.int32).reshape(T, -1)
    assert (rep[:, 0] == 0).all() or (np.isin(rep[:, 0], [0, 4])).all(), "batch reported errors"
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # per-stage times from further calls with the library's stage events (not part of the timed steps)
    nst = len(simulee.STAGES)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nst)] for _ in range(3)]
    for row in sev:
        for e in row:
            e.record(stream)
    for row in sev:
        chk.set_stage_events(row)
        call()
    torch.cuda.synchronize()
    chk.set_stage_events(None)
    stage_ms = {name: sum(r[2 * k].elapsed_time(r[2 * k + 1]) for r in sev) / len(sev)
                for k, name in enumerate(simulee.STAGES)}
    # the same call captured once in a CUDA graph and replayed
    g = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream()
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        stream = s2
        with torch.cuda.graph(g, stream=s2):
            call()
    stream = torch.cuda.current_stream()
    g.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_g = e0.elapsed_time(e1) / args.steps
    n_ev = sum(d.n_events for d in dts)
    return {"workload": f"batch: {T} traces, lognormal sizes (median 1e5, sigma 0.87, clipped 1e3..1e7), "
                        f"block sizes 64..1024, 4..64 epochs", "traces": T, "n_events": n_ev,
            "value": n_ev / (ms * 1e-3) / 1e9, "ms_per_step": ms,
            "graph_value": n_ev / (ms_g * 1e-3) / 1e9, "graph_ms_per_step": ms_g, "unit": UNIT,
            "stages_ms": stage_ms,
            "launches_per_step": chk.last_launches(), "workspace_bytes": ws.numel(), "gen_s": gen_s,
            **({"cpu_baseline": base} if base else {})}


def _oracle_trace_worker(job):
    """One batch member checked by the oracle (runs in a spawned process; generation not timed)."""
    import oracle
    import tracegen
    i, n, bs, ep = job
    tr = tracegen.c3_trace(i, n, bs, ep)
    t0 = time.perf_counter()
    out = oracle.check(tr)
    assert out["status"] == 0
    return tr.n_events, time.perf_counter() - t0


def batch_oracle_baseline(sizes, bss, eps, stride: int = 32) -> dict:
    """The oracle over every stride-th batch member, one process per host core (spawned before any GPU work)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    jobs = [(i, int(sizes[i]), int(bss[i]), int(eps[i])) for i in range(0, len(sizes), stride)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_trace_worker, jobs[:cores])        # warm-up: load the oracle in every worker
        t0 = time.perf_counter()
        res = pool.map(_oracle_trace_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    n = sum(r[0] for r in res)
    return {"value": n / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {stride}th batch member ({len(jobs)} traces, {n} records), one process per core, "
                      f"{wall:.1f} s wall"}


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
    chk = simulee.Checker(0)
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
            "results": {"status": r.status, "n_races": r.n_races, "n_divergence": r.n_divergence,
                        "n_redundant": r.n_redundant, "n_grid_redundant": r.n_grid_redundant}}
    if not args.no_cpu_baseline:
        n, secs = run_oracle_sample(tr, sample_blocks)
        line["cpu_baseline"] = {"value": n / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"records of blocks 0..{sample_blocks - 1} ({n} records, {secs:.2f} s)"}
    return line


def fitness_arm(args):
    """Fitness of Eq. 1 (distinct addresses / distinct address-thread pairs) over the grid workload: records
    per second through simulee_fitness_batch, with the radix plan's algorithmic bytes against the HBM peak."""
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
    # key bits: gtid + unit + block + space (one trace): radix passes of 8 bits, 8-byte keys when wider than 32 bits
    kb = bits(tr.n_blocks * tr.block_threads) + bits(max(tr.shared_units, tr.global_units)) + bits(tr.n_blocks) + 1
    npass, kw = -(-kb // 8), (8 if kb > 32 else 4)
    n = tr.n_events
    algo = n * (16 + kw + 2 * npass * kw + kw) + 4 * tr.barrier_counts.size   # read, key write, passes, count
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


def serve_arm(args):
    """Serving workload: Poisson arrivals of check jobs, sizes log-uniform 1e4..1e8 records from the
    grid and barrier generators, continuous batching under a 120 GB HBM budget, against serial checking."""
    import torch
    import tracegen
    from paper_1905_01833_gb300 import serve
    rng = np.random.default_rng(7)
    pool_sizes = np.exp(np.linspace(np.log(1e4), np.log(1e8), args.serve_pool))
    trs = []
    for i, sz in enumerate(pool_sizes):
        if i % 2 == 0:   # grid family: 256-thread blocks, 32 epochs (~2e5 records per block)
            nb = max(1, int(round(sz / 59600)))
            tr = tracegen.pattern(100 + i, n_blocks=nb, block_threads=256, n_epochs=32, shared_units=12288,
                                  global_units=1 << max(20, int(np.ceil(np.log2(4096 + 2 * 1024 * nb)))))
            if tr.n_events > sz:
                tr.events = np.ascontiguousarray(tr.events[:int(sz)])
        else:            # barrier family: 1024-thread blocks, 64 epochs, 4 accesses (262144 records per block)
            nb = max(1, int(round(sz / 262144)))
            tr = tracegen.barrier(100 + i, n_blocks=nb, block_threads=1024, n_epochs=64, shared_units=8192)
            if tr.n_events > sz:
                tr.events = np.ascontiguousarray(tr.events[:int(sz)])
        trs.append(tr)
    dts, keep = device_pool(torch, trs, "cuda:0")
    del trs
    draws = np.exp(rng.uniform(np.log(1e4), np.log(1e8), size=args.serve_jobs))
    pick = np.abs(np.log(draws)[:, None] - np.log(pool_sizes)[None, :]).argmin(axis=1)

    def run(rate, serial):
        arr = serve.poisson_arrivals(rate, args.serve_jobs, seed=11)
        jobs = [serve.Job(i, dts[int(pick[i])], float(arr[i])) for i in range(args.serve_jobs)]
        srv = serve.Server(0, hbm_budget=120 << 30, serial=serial, keep_lists=False)
        return srv.run(jobs)

    warm = serve.Server(0, keep_lists=False)
    warm.run([serve.Job(i, dts[i % len(dts)], 0.0) for i in range(len(dts))])
    res = {"workload": f"serve: Poisson arrivals, {args.serve_jobs} jobs, sizes log-uniform 1e4..1e8 records "
                       f"(pool of {len(dts)} device-resident traces), 120 GB budget",
           "unit": UNIT, "rates": {}}
    for rate in args.serve_rates:
        a = run(rate, serial=False)
        b = run(rate, serial=True)
        res["rates"][str(rate)] = {
            "batched": {k: a[k] for k in ("p50_ms", "p99_ms", "max_ms", "batches", "max_batch", "max_inflight")}
            | {"value": a["events_per_s"] / 1e9},
            "serial": {k: b[k] for k in ("p50_ms", "p99_ms", "max_ms")} | {"value": b["events_per_s"] / 1e9}}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", choices=["auto", "sort"], default="auto")
    ap.add_argument("--hash-shape", type=int, choices=[0, 1, 2], default=0,
                    help="hash path CTAs: 0 chosen per call, 1 one 1024-thread CTA per SM, 2 two 512-thread CTAs")
    ap.add_argument("--graph-replay", choices=["auto", "off"], default="auto",
                    help="auto: repeated identical calls replayed by the library as one CUDA graph; off: direct launches")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--oracle-blocks", type=int, default=256)
    ap.add_argument("--ref-blocks", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--blocks", type=int, default=1024, help="grid blocks (1024 = the benchmark workload; "
                    "smaller values only for profiling captures)")
    ap.add_argument("--workload", choices=["grid", "batch", "serve", "fitness", "evolve", "strided", "barrier", "warp",
                                           "paper"],
                    default="grid",
                    help="grid: the benchmark line; batch / serve: the batched and served forms; fitness: Eq. 1 "
                         "over the grid workload (separate lines)")
    ap.add_argument("--batch-traces", type=int, default=4096)
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 1000.0, 4000.0])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload != "grid" and args.impl == "ours":
        import torch
        torch.cuda.set_device(0)
        out = {"batch": batch_arm, "serve": serve_arm, "fitness": fitness_arm, "evolve": evolve_arm,
               "strided": single_trace_arm, "barrier": single_trace_arm, "warp": single_trace_arm,
               "paper": single_trace_arm}[args.workload](args)
        print(json.dumps({"metric": METRIC, **out}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    from paper_1905_01833_gb300 import simulee
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    tr = make_trace(rank, args.blocks)
    dt = simulee.to_device(tr, f"cuda:{local}")
    chk = simulee.Checker(local, path=simulee.PATH_SORT if args.path == "sort" else simulee.PATH_AUTO,
                          hash_shape=args.hash_shape,
                          graph_replay=simulee.GRAPH_OFF if args.graph_replay == "off" else simulee.GRAPH_AUTO)
    ws = chk.workspace(chk.workspace_size(dt))
    caps = dict(races_cap=4_000_000, div_cap=tr.n_blocks, red_cap=tr.n_blocks * tr.max_barriers,
                grid_cap=tr.max_barriers)
    outs, bufs = chk.alloc_outputs(caps["races_cap"], caps["div_cap"], caps["red_cap"], caps["grid_cap"])
    report_dev = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    L = simulee.lib()
    ctrace = dt.c()
    import ctypes
    sp = ctypes.c_void_p(stream.cuda_stream)

    def step(trace_c, rep_ptr):
        s = L.simulee_check(chk.h, ctypes.byref(trace_c), ctypes.byref(outs), ctypes.c_void_p(rep_ptr),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), sp)
        if s != 0:
            raise RuntimeError(f"simulee_check failed: {simulee.status_str(s)}")

    for _ in range(args.warmup):
        step(ctrace, report_dev.data_ptr())
    torch.cuda.synchronize()
    rep0 = simulee.Report.from_buffer_copy(report_dev.cpu().numpy().tobytes())
    if rep0.status != 0:
        raise RuntimeError(f"check reported status {rep0.status}")
    launches = chk.last_launches()

    # stage events for every timed step
    nst = len(simulee.STAGES)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * nst)] for _ in range(args.steps)]
    for row in evs:
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_uuid(torch, local) if world == 1 else None)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        step(ctrace, report_dev.data_ptr())
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = t_start.elapsed_time(t_end) / args.steps
    # per-stage times from a second run of the same steps with stage events (not the timed steps above,
    # so the events add nothing to their time)
    for i in range(args.steps):
        chk.set_stage_events(evs[i])
        step(ctrace, report_dev.data_ptr())
    torch.cuda.synchronize()
    chk.set_stage_events(None)
    stage_ms = {name: sum(evs[i][2 * s].elapsed_time(evs[i][2 * s + 1]) for i in range(args.steps)) / args.steps
                for s, name in enumerate(simulee.STAGES)}
    # the same steps with graph replay off: every call issues its kernels one by one
    direct = None
    if world == 1:
        chk_d = simulee.Checker(local, path=simulee.PATH_SORT if args.path == "sort" else simulee.PATH_AUTO,
                                hash_shape=args.hash_shape, graph_replay=simulee.GRAPH_OFF)

        def step_d():
            s = L.simulee_check(chk_d.h, ctypes.byref(ctrace), ctypes.byref(outs), ctypes.c_void_p(report_dev.data_ptr()),
                                ctypes.c_void_p(ws.data_ptr()), ws.numel(), sp)
            if s != 0:
                raise RuntimeError(f"simulee_check failed: {simulee.status_str(s)}")
        for _ in range(3):
            step_d()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            step_d()
        g1.record(stream)
        torch.cuda.synchronize()
        ms_d = g0.elapsed_time(g1) / args.steps
        direct = {"value": tr.n_events / (ms_d * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_d,
                  "launches_per_step": chk_d.last_launches()}
        chk_d.close()
    rep = simulee.Report.from_buffer_copy(report_dev.cpu().numpy().tobytes())
    assert rep.status == 0 and rep.n_races == rep0.n_races and rep.n_redundant == rep0.n_redundant

    value, ms = job_value(tr.n_events, ms, dist, f"cuda:{local}")

    # end to end through the C ABI: pinned host trace -> device, check, report and lists -> host, every
    # step. Two device trace buffers: the next step's records go up on a copy stream while this step
    # is checked (one context per buffer, so that each keeps its own replay graph); the same steps
    # one after another give e2e_serial.
    h_ev = torch.from_numpy(tr.events.view(np.int32)).pin_memory()
    h_cn = torch.from_numpy(tr.barrier_counts.view(np.int32)).pin_memory()
    d_ev = [torch.empty_like(dt.events) for _ in range(2)]
    d_cn = [torch.empty_like(dt.barrier_counts) for _ in range(2)]
    etr = [simulee.DeviceTrace(d_ev[q], d_cn[q], tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units,
                               tr.max_barriers).c() for q in range(2)]
    chks = [chk, simulee.Checker(local, path=simulee.PATH_SORT if args.path == "sort" else simulee.PATH_AUTO,
                                 hash_shape=args.hash_shape,
                                 graph_replay=simulee.GRAPH_OFF if args.graph_replay == "off" else simulee.GRAPH_AUTO)]
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
            copy_s.wait_event(freed[q])   # the check of step i - 2 has read this buffer
        with torch.cuda.stream(copy_s):
            d_ev[q].copy_(h_ev, non_blocking=True)
            d_cn[q].copy_(h_cn, non_blocking=True)
        copied[q].record(copy_s)

    def finish_step(i):
        nonlocal d2h
        q = i % 2
        stream.wait_event(copied[q])
        s_ = L.simulee_check(chks[q].h, ctypes.byref(etr[q]), ctypes.byref(outs), ctypes.c_void_p(rep_host.data_ptr()),
                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), sp)
        if s_ != 0:
            raise RuntimeError(f"simulee_check failed: {simulee.status_str(s_)}")
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
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_e2e(args.e2e_steps, True)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_value, _ = job_value(tr.n_events, e2e_s * 1e3, dist, f"cuda:{local}")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_e2e(max(2, args.e2e_steps // 2), False)
    e2e_serial_s = (time.perf_counter() - t0) / max(2, args.e2e_steps // 2)
    e2e_serial, _ = job_value(tr.n_events, e2e_serial_s * 1e3, dist, f"cuda:{local}")
    chks[1].close()
    h2d = tr.events.nbytes + tr.barrier_counts.nbytes

    # roofline of the dominant stage
    sizes = chk.stream_sizes()
    sb = stage_bytes(tr, sizes, args.path, *global_counts(tr))
    peak, peak_src = peaks()
    cand = [k for k in ("ingest", "hash", "fallback", "sort", "reduce") if sb[k] > 0]
    dom = max(cand, key=lambda k: stage_ms[k])
    kname = {"ingest": "k_ingest", "hash": "k_hash_blocks", "fallback": "k_ingest", "sort": "k_onesweep",
             "reduce": "k_reduce_groups"}[dom]
    nl = sb["launches"][dom]
    achieved = sb[dom] / (stage_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "bytes_per_launch": sb[dom] / nl, "launch_ms": stage_ms[dom] / nl,
                "traffic": kernel_traffic(kname, "grid")}
    stage_gbs = {k: sb[k] / (stage_ms[k] * 1e-3) / 1e9 for k in cand if stage_ms[k] > 0}
    # the whole plan: algorithmic bytes per record over every stage, and the single-read floor (16 B per record)
    b_plan = sum(sb[k] for k in ("ingest", "hash", "fallback", "sort", "reduce")) / tr.n_events
    roofline["plan"] = {"bytes_per_record": b_plan, "frac": value * 1e9 * b_plan / (peak * 1e9),
                        "floor_frac": value * 1e9 * 16 / (peak * 1e9),
                        "radix_passes": sb["launches"]["sort"] - 1}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.blocks == 1024 else WORKLOAD.replace("1024 blocks", f"{args.blocks} blocks"),
                   "n_events": tr.n_events, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (1 GB trace, 129 MB L2); no flush", "path": args.path},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "serial_value": e2e_serial,
                "overlap": "two device trace buffers: the next step's host-to-device copy runs on a copy "
                           "stream while the current step is checked; serial_value = copy, check and "
                           "read-back one after another"},
        "gpu_launches": launches * args.steps,
        "launch": "repeated identical calls replayed by the library as one CUDA graph (graph_replay auto); "
                  "'direct' times the same steps with every kernel launched by the call",
        "direct": direct,
        "roofline": roofline,
        "stages_ms": stage_ms,
        "stages_gbs": stage_gbs,
        "streams": sizes,
        "results": {"n_races": rep.n_races, "n_divergence": rep.n_divergence, "n_redundant": rep.n_redundant,
                    "n_grid_redundant": rep.n_grid_redundant},
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, secs = run_oracle_sample(tr, args.oracle_blocks)
        line["cpu_baseline"] = {"value": n / secs / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"records of blocks 0..{args.oracle_blocks - 1} of the same trace "
                                          f"({n} records, {secs:.1f} s, single thread)",
                                "host_cores": len(os.sched_getaffinity(0))}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
