"""Python binding of the C ABI in include/simulee.h (argument marshalling only).

Every step of the check runs in the CUDA library (libsimulee.so). PyTorch
supplies device memory and the current CUDA stream. If the library is missing
the calls raise; there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimulee.so")

OK, EINVAL, EBADTRACE, ENOMEM, ETRUNC, ETIMEOUT, ECUDA = range(7)
FLAG_UNSORTED = 1
FLAG_WARP_AWARE = 2
FLAG_PAPER_ORDER = 4   # the paper's visit-order counters (Algorithm 3) group the tuples
STMT_DIVERGED = 0x80000000
PATH_AUTO, PATH_SORT, PATH_HASH = 0, 1, 2
GRAPH_AUTO, GRAPH_OFF = 0, 1   # repeated identical check calls replayed as one CUDA graph, or always direct
STAGES = ("ingest", "sort", "reduce", "races", "blocks", "hash", "fallback")

RACE_DTYPE = np.dtype([("space", "u1"), ("scope", "u1"), ("cls", "u1"), ("pad", "u1"),
                       ("block", "<u4"), ("epoch", "<u4"), ("unit", "<u4"),
                       ("vo_first", "<u4"), ("vo_second", "<u4"),
                       ("gtid_first", "<u4"), ("gtid_second", "<u4")])
DIV_DTYPE = np.dtype([("block", "<u4"), ("min_count", "<u4"), ("max_count", "<u4"), ("first_min_tid", "<u4")])
BAR_DTYPE = np.dtype([("block", "<u4"), ("barrier", "<u4")])


class SimuleeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


class Trace(ctypes.Structure):
    _fields_ = [("events", ctypes.c_void_p), ("n_events", ctypes.c_uint64), ("barrier_counts", ctypes.c_void_p),
                ("n_blocks", ctypes.c_uint32), ("block_threads", ctypes.c_uint32), ("shared_units", ctypes.c_uint32),
                ("global_units", ctypes.c_uint32), ("max_barriers", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("stmt", ctypes.c_void_p)]


class Outputs(ctypes.Structure):
    _fields_ = [("races", ctypes.c_void_p), ("races_cap", ctypes.c_uint64),
                ("divergence", ctypes.c_void_p), ("divergence_cap", ctypes.c_uint64),
                ("redundant", ctypes.c_void_p), ("redundant_cap", ctypes.c_uint64),
                ("grid_redundant", ctypes.c_void_p), ("grid_redundant_cap", ctypes.c_uint64)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("bad_kind", ctypes.c_uint32), ("bad_index", ctypes.c_uint64),
                ("n_races", ctypes.c_uint64), ("n_divergence", ctypes.c_uint64), ("n_redundant", ctypes.c_uint64),
                ("n_grid_redundant", ctypes.c_uint64)]


class Options(ctypes.Structure):
    _fields_ = [("wait_limit_us", ctypes.c_uint32), ("path", ctypes.c_uint32), ("test_withhold", ctypes.c_uint32),
                ("ingest_ctas_per_sm", ctypes.c_uint32), ("sort_ctas_per_sm", ctypes.c_uint32),
                ("reduce_ctas_per_sm", ctypes.c_uint32), ("hash_shape", ctypes.c_uint32), ("graph_replay", ctypes.c_uint32),
                ("sort_items", ctypes.c_uint32), ("radix_bits", ctypes.c_uint32), ("hash_cap_eighths", ctypes.c_uint32),
                ("hash_pool_div", ctypes.c_uint32), ("hot_unit_marks", ctypes.c_uint32),
                ("hash_groups", ctypes.c_uint32)]


class Fitness(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("bad_kind", ctypes.c_uint32), ("bad_index", ctypes.c_uint64),
                ("n_addresses", ctypes.c_uint64), ("n_pairs", ctypes.c_uint64),
                ("shared_lo", ctypes.c_uint32), ("shared_hi", ctypes.c_uint32),
                ("global_lo", ctypes.c_uint32), ("global_hi", ctypes.c_uint32)]


class Model(ctypes.Structure):
    _fields_ = [("model", ctypes.c_uint32), ("grid_x", ctypes.c_uint32), ("grid_y", ctypes.c_uint32),
                ("block_x", ctypes.c_uint32), ("block_y", ctypes.c_uint32), ("arg0", ctypes.c_int32),
                ("arg1", ctypes.c_int32), ("reserved", ctypes.c_uint32), ("events_off", ctypes.c_uint64),
                ("counts_off", ctypes.c_uint64)]


MODEL_COPY2D, MODEL_STENCIL = 0, 1
MODEL_SHARED_UNITS, MODEL_GLOBAL_UNITS = 4096, 1 << 20

REPORT_BYTES = ctypes.sizeof(Report)
FITNESS_BYTES = ctypes.sizeof(Fitness)
_lib_handle = None


def lib():
    """Load libsimulee.so; raise if it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, st = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        P = ctypes.POINTER
        sigs = {
            "simulee_create": [P(vp), ctypes.c_int, P(Options)],
            "simulee_destroy": [vp],
            "simulee_workspace_size": [vp, P(Trace), P(ctypes.c_size_t)],
            "simulee_check": [vp, P(Trace), P(Outputs), vp, vp, ctypes.c_size_t, vp],
            "simulee_check_races": [vp, P(Trace), vp, u64, vp, vp, ctypes.c_size_t, vp],
            "simulee_check_divergence": [vp, P(Trace), vp, u64, vp, vp, ctypes.c_size_t, vp],
            "simulee_check_redundant_barriers": [vp, P(Trace), vp, u64, vp, u64, vp, vp, ctypes.c_size_t, vp],
            "simulee_batch_workspace_size": [vp, P(Trace), u32, P(ctypes.c_size_t)],
            "simulee_check_batch": [vp, P(Trace), u32, P(Outputs), vp, vp, ctypes.c_size_t, vp],
        }
        sigs["simulee_set_stage_events"] = [vp, P(vp), u32]
        sigs["simulee_compact_workspace_size"] = [vp, P(Trace), u32, P(ctypes.c_size_t)]
        sigs["simulee_check_noalloc"] = [vp, P(Trace), P(Outputs), vp, vp]
        sigs["simulee_stream_sizes"] = [vp, vp, vp, vp]
        sigs["simulee_hash_groups"] = [vp, vp, vp, vp]
        sigs["simulee_fitness_workspace_size"] = [vp, P(Trace), u32, P(ctypes.c_size_t)]
        sigs["simulee_fitness_batch"] = [vp, P(Trace), u32, vp, vp, ctypes.c_size_t, vp]
        sigs["simulee_model_traces"] = [vp, vp, u32, vp, u64, vp, u64, vp]
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        L.simulee_last_launches.argtypes = [vp]
        L.simulee_last_launches.restype = u32
        L.simulee_last_replayed.argtypes = [vp]
        L.simulee_last_replayed.restype = u32
        L.simulee_status_str.argtypes = [st]
        L.simulee_status_str.restype = ctypes.c_char_p
        _lib_handle = L
    return _lib_handle


def status_str(s: int) -> str:
    return lib().simulee_status_str(s).decode()


def _check(s: int, what: str):
    if s != OK:
        raise SimuleeError(s, f"{what}: {status_str(s)}")


@dataclasses.dataclass
class DeviceTrace:
    """A trace whose records and barrier counts live in device memory (torch tensors)."""
    events: object          # torch.int32 (n, 4) on cuda
    barrier_counts: object  # torch.int32 (n_blocks * block_threads,) on cuda
    n_blocks: int
    block_threads: int
    shared_units: int
    global_units: int
    max_barriers: int
    flags: int = 0
    stmt: object = None     # torch.int32 (n,) on cuda: statement words of a warp-aware trace

    @property
    def n_events(self) -> int:
        return int(self.events.shape[0])

    def c(self) -> Trace:
        st = self.stmt.data_ptr() if (self.stmt is not None and self.n_events) else None
        return Trace(self.events.data_ptr() if self.n_events else None, self.n_events,
                     self.barrier_counts.data_ptr(), self.n_blocks, self.block_threads, self.shared_units,
                     self.global_units, self.max_barriers, self.flags, st)


def to_device(trace, device="cuda") -> DeviceTrace:
    """Copy a host trace (numpy arrays + dimensions) to the GPU."""
    import torch
    ev = torch.from_numpy(np.ascontiguousarray(trace.events, dtype=np.uint32).view(np.int32).reshape(-1, 4))
    cn = torch.from_numpy(np.ascontiguousarray(trace.barrier_counts, dtype=np.uint32).view(np.int32))
    st = getattr(trace, "stmt", None)
    st = None if st is None else torch.from_numpy(np.ascontiguousarray(st, dtype=np.uint32).view(np.int32)).to(device)
    return DeviceTrace(ev.to(device), cn.to(device), trace.n_blocks, trace.block_threads, trace.shared_units,
                       trace.global_units, trace.max_barriers, getattr(trace, "flags", 0), st)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Checker:
    """A library context on one GPU plus reusable device buffers."""

    def __init__(self, device: int = 0, wait_limit_us: int = 0, path: int = PATH_AUTO, test_withhold: int = 0,
                 ingest_ctas_per_sm: int = 0, sort_ctas_per_sm: int = 0, reduce_ctas_per_sm: int = 0,
                 hash_shape: int = 0, graph_replay: int = GRAPH_AUTO, sort_items: int = 0, radix_bits: int = 0,
                 hash_cap_eighths: int = 0, hash_pool_div: int = 0, hot_unit_marks: int = 0, hash_groups: int = 0):
        import torch
        self.device = device
        self.torch = torch
        opt = Options(wait_limit_us, path, test_withhold, ingest_ctas_per_sm, sort_ctas_per_sm, reduce_ctas_per_sm,
                      hash_shape, graph_replay, sort_items, radix_bits, hash_cap_eighths, hash_pool_div,
                      hot_unit_marks, hash_groups)
        h = ctypes.c_void_p()
        _check(lib().simulee_create(ctypes.byref(h), device, ctypes.byref(opt)), "simulee_create")
        self.h = h
        self._ws = None
        self._report = torch.zeros(REPORT_BYTES, dtype=torch.uint8).pin_memory()

    def close(self):
        if self.h:
            lib().simulee_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_launches(self) -> int:
        """Kernels launched by the last check call."""
        return int(lib().simulee_last_launches(self.h))

    def last_replayed(self) -> bool:
        """The last check call was issued as one CUDA graph launch (graph replay)."""
        return bool(lib().simulee_last_replayed(self.h))

    def set_stage_events(self, events) -> None:
        """Record the given timing events around the check's stages (2 per stage); None turns it off."""
        if not events:
            _check(lib().simulee_set_stage_events(self.h, None, 0), "simulee_set_stage_events")
            return
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        _check(lib().simulee_set_stage_events(self.h, arr, len(events)), "simulee_set_stage_events")

    def stream_sizes(self, stream=None) -> dict:
        """Record counts that the last check on this checker's workspace sent through the radix sort."""
        out = self.torch.zeros(5, dtype=self.torch.int32, device=f"cuda:{self.device}")
        _check(lib().simulee_stream_sizes(self.h, ctypes.c_void_p(self._ws.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          _stream_ptr(stream)), "simulee_stream_sizes")
        v = [int(x) for x in out.cpu().tolist()]
        # x_slots: inter-block stream slots written (global records, plus unused reserved slots on the hash path)
        return dict(n_s=v[0], n_g=v[1], n_x=v[2], n_races=v[3], x_slots=v[4])

    def hash_groups(self, stream=None) -> dict:
        """Blocks per hash-path launch group in the last check on this checker's workspace: checked by
        128-thread groups (quarter), 256-thread groups (half), whole smaller CTAs (small), larger CTAs (large)."""
        out = self.torch.zeros(5, dtype=self.torch.int32, device=f"cuda:{self.device}")
        _check(lib().simulee_hash_groups(self.h, ctypes.c_void_p(self._ws.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         _stream_ptr(stream)), "simulee_hash_groups")
        v = [int(x) for x in out.cpu().tolist()]
        return dict(zip(("quarter", "half", "small", "large"), (v[i + 1] - v[i] for i in range(4))))

    def workspace_size(self, dt: DeviceTrace) -> int:
        n = ctypes.c_size_t()
        t = dt.c()
        _check(lib().simulee_workspace_size(self.h, ctypes.byref(t), ctypes.byref(n)), "simulee_workspace_size")
        return int(n.value)

    def compact_workspace_size(self, dts) -> int:
        """Compact workspace bytes for a call over these traces (a list; one trace for the single-trace calls)."""
        arr = (Trace * len(dts))(*[d.c() for d in dts])
        n = ctypes.c_size_t()
        _check(lib().simulee_compact_workspace_size(self.h, arr, len(dts), ctypes.byref(n)),
               "simulee_compact_workspace_size")
        return int(n.value)

    def workspace(self, nbytes: int):
        """A device workspace of at least nbytes, reused across calls (256-byte aligned)."""
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = self.torch.empty(max(nbytes, 256), dtype=self.torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    def alloc_outputs(self, races_cap: int, div_cap: int, red_cap: int, grid_cap: int):
        torch = self.torch
        dev = f"cuda:{self.device}"
        bufs = dict(races=torch.empty(max(races_cap, 1) * 32, dtype=torch.uint8, device=dev),
                    divergence=torch.empty(max(div_cap, 1) * 16, dtype=torch.uint8, device=dev),
                    redundant=torch.empty(max(red_cap, 1) * 8, dtype=torch.uint8, device=dev),
                    grid=torch.empty(max(grid_cap, 1) * 4, dtype=torch.uint8, device=dev))
        o = Outputs(bufs["races"].data_ptr(), races_cap, bufs["divergence"].data_ptr(), div_cap,
                    bufs["redundant"].data_ptr(), red_cap, bufs["grid"].data_ptr(), grid_cap)
        return o, bufs

    def report(self) -> dict:
        r = Report.from_buffer_copy(self._report.numpy().tobytes())
        return dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                    n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)

    def check(self, dt: DeviceTrace, races_cap: int | None = None, div_cap: int | None = None,
              red_cap: int | None = None, grid_cap: int | None = None, stream=None, compact: bool = False) -> dict:
        """Full check; returns the report plus host copies of the (truncated) lists. compact: a workspace of
        simulee_compact_workspace_size bytes (the report says ENOMEM if the call needed more)."""
        torch = self.torch
        n = dt.n_events
        races_cap = 2 * n + 2 if races_cap is None else races_cap
        div_cap = dt.n_blocks if div_cap is None else div_cap
        red_cap = dt.n_blocks * max(dt.max_barriers, 1) if red_cap is None else red_cap
        grid_cap = max(dt.max_barriers, 1) if grid_cap is None else grid_cap
        o, bufs = self.alloc_outputs(races_cap, div_cap, red_cap, grid_cap)
        need = self.compact_workspace_size([dt]) if compact else self.workspace_size(dt)
        ws = self.workspace(need)
        t = dt.c()
        _check(lib().simulee_check(self.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(self._report.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), need, _stream_ptr(stream)), "simulee_check")
        torch.cuda.synchronize(self.device)
        rep = self.report()
        return self._collect(rep, bufs, races_cap, div_cap, red_cap, grid_cap)

    def _collect(self, rep, bufs, races_cap, div_cap, red_cap, grid_cap):
        def take(buf, cap, count, dtype):
            k = min(cap, count) if rep["status"] in (OK, ETRUNC) else 0
            return np.frombuffer(buf[: k * dtype.itemsize].cpu().numpy().tobytes(), dtype=dtype)
        out = dict(rep)
        out["races"] = take(bufs["races"], races_cap, rep["n_races"], RACE_DTYPE)
        out["divergence"] = take(bufs["divergence"], div_cap, rep["n_divergence"], DIV_DTYPE)
        out["redundant"] = take(bufs["redundant"], red_cap, rep["n_redundant"], BAR_DTYPE)
        out["grid_redundant"] = take(bufs["grid"], grid_cap, rep["n_grid_redundant"], np.dtype("<u4"))
        return out

    def batch_workspace_size(self, dts) -> int:
        arr = (Trace * len(dts))(*[d.c() for d in dts])
        n = ctypes.c_size_t()
        _check(lib().simulee_batch_workspace_size(self.h, arr, len(dts), ctypes.byref(n)),
               "simulee_batch_workspace_size")
        return int(n.value)

    def model_traces(self, launches, stream=None) -> list:
        """Traces of model-kernel launches, generated on the device.

        launches: sequence of (model, (grid_x, grid_y), (block_x, block_y), (arg0, arg1)) with integer
        arguments. Returns DeviceTrace views into two shared device buffers."""
        torch = self.torch
        T = len(launches)
        ms = (Model * T)()
        ev_off = ct_off = 0
        dims = []
        for i, (model, grid, block, args) in enumerate(launches):
            nb, bt = grid[0] * grid[1], block[0] * block[1]
            ne = nb * bt * (2 if model == MODEL_COPY2D else 3)
            ms[i] = Model(model, grid[0], grid[1], block[0], block[1], int(args[0]), int(args[1]), 0, ev_off, ct_off)
            dims.append((ev_off, ne, ct_off, nb, bt, model))
            ev_off += ne
            ct_off += nb * bt
        dev = f"cuda:{self.device}"
        m_dev = torch.from_numpy(np.frombuffer(bytes(ms), dtype=np.uint8).copy()).to(dev)
        ev = torch.empty((max(ev_off, 1), 4), dtype=torch.int32, device=dev)
        cn = torch.empty(max(ct_off, 1), dtype=torch.int32, device=dev)
        _check(lib().simulee_model_traces(self.h, ctypes.c_void_p(m_dev.data_ptr()), T, ctypes.c_void_p(ev.data_ptr()),
                                          ev_off, ctypes.c_void_p(cn.data_ptr()), ct_off, _stream_ptr(stream)),
               "simulee_model_traces")
        out = []
        for (eo, ne, co, nb, bt, model) in dims:
            out.append(DeviceTrace(ev[eo:eo + ne], cn[co:co + nb * bt], nb, bt, MODEL_SHARED_UNITS,
                                   MODEL_GLOBAL_UNITS, 0 if model == MODEL_COPY2D else 1))
        self._model_bufs = (m_dev, ev, cn)   # keep the buffers alive with the views
        return out

    def fitness_workspace_size(self, dts) -> int:
        T = len(dts)
        arr = (Trace * T)(*[d.c() for d in dts])
        n = ctypes.c_size_t()
        _check(lib().simulee_fitness_workspace_size(self.h, arr, T, ctypes.byref(n)), "simulee_fitness_workspace_size")
        return int(n.value)

    def fitness_batch(self, dts, stream=None) -> list[dict]:
        """Eq. 1 fitness of each trace: sum g, sum f (F = n_addresses / n_pairs) and the unit ranges."""
        torch = self.torch
        T = len(dts)
        out = torch.zeros(T * FITNESS_BYTES, dtype=torch.uint8, device=f"cuda:{self.device}")
        arr = (Trace * T)(*[d.c() for d in dts])
        ws = self.workspace(self.fitness_workspace_size(dts))
        _check(lib().simulee_fitness_batch(self.h, arr, T, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)),
               "simulee_fitness_batch")
        torch.cuda.synchronize(self.device)
        raw = out.cpu().numpy().tobytes()
        res = []
        for i in range(T):
            f = Fitness.from_buffer_copy(raw[i * FITNESS_BYTES:(i + 1) * FITNESS_BYTES])
            res.append({name: int(getattr(f, name)) for name, _ in Fitness._fields_})
        return res

    def check_batch(self, dts, races_caps=None, stream=None, compact: bool = False) -> list[dict]:
        """Check independent traces in one batched call; returns one result dict per trace. compact: a
        workspace of simulee_compact_workspace_size bytes."""
        torch = self.torch
        T = len(dts)
        dev = f"cuda:{self.device}"
        rc = [2 * d.n_events + 2 for d in dts] if races_caps is None else list(races_caps)
        dc = [d.n_blocks for d in dts]
        bc = [d.n_blocks * max(d.max_barriers, 1) for d in dts]
        gc = [max(d.max_barriers, 1) for d in dts]
        sizes = {"races": (rc, 32), "divergence": (dc, 16), "redundant": (bc, 8), "grid": (gc, 4)}
        bufs, offs = {}, {}
        for k, (caps, w) in sizes.items():
            o = np.concatenate([[0], np.cumsum([c * w for c in caps])]).astype(np.int64)
            offs[k] = o
            bufs[k] = torch.empty(max(int(o[-1]), 16), dtype=torch.uint8, device=dev)
        outs = (Outputs * T)()
        for i in range(T):
            outs[i] = Outputs(bufs["races"].data_ptr() + int(offs["races"][i]), rc[i],
                              bufs["divergence"].data_ptr() + int(offs["divergence"][i]), dc[i],
                              bufs["redundant"].data_ptr() + int(offs["redundant"][i]), bc[i],
                              bufs["grid"].data_ptr() + int(offs["grid"][i]), gc[i])
        reports = torch.zeros(T * REPORT_BYTES, dtype=torch.uint8, device=dev)
        arr = (Trace * T)(*[d.c() for d in dts])
        need = self.compact_workspace_size(dts) if compact else self.batch_workspace_size(dts)
        ws = self.workspace(need)
        _check(lib().simulee_check_batch(self.h, arr, T, outs, ctypes.c_void_p(reports.data_ptr()),
                                         ctypes.c_void_p(ws.data_ptr()), need, _stream_ptr(stream)),
               "simulee_check_batch")
        torch.cuda.synchronize(self.device)
        rep_bytes = reports.cpu().numpy().tobytes()
        host = {k: v.cpu().numpy() for k, v in bufs.items()}
        res = []
        for i in range(T):
            r = Report.from_buffer_copy(rep_bytes[i * REPORT_BYTES:(i + 1) * REPORT_BYTES])
            rep = dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                       n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)
            ok = rep["status"] in (OK, ETRUNC)

            def take(kind, cap, count, dtype):
                k = min(cap, count) if ok else 0
                o = int(offs[kind][i])
                return np.frombuffer(host[kind][o:o + k * dtype.itemsize].tobytes(), dtype=dtype)
            rep["races"] = take("races", rc[i], rep["n_races"], RACE_DTYPE)
            rep["divergence"] = take("divergence", dc[i], rep["n_divergence"], DIV_DTYPE)
            rep["redundant"] = take("redundant", bc[i], rep["n_redundant"], BAR_DTYPE)
            rep["grid_redundant"] = take("grid", gc[i], rep["n_grid_redundant"], np.dtype("<u4"))
            res.append(rep)
        return res

    def check_races(self, dt: DeviceTrace, cap: int | None = None, stream=None) -> dict:
        cap = 2 * dt.n_events + 2 if cap is None else cap
        o, bufs = self.alloc_outputs(cap, 0, 0, 0)
        ws = self.workspace(self.workspace_size(dt))
        t = dt.c()
        _check(lib().simulee_check_races(self.h, ctypes.byref(t), ctypes.c_void_p(o.races), cap,
                                         ctypes.c_void_p(self._report.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                         ws.numel(), _stream_ptr(stream)), "simulee_check_races")
        self.torch.cuda.synchronize(self.device)
        return self._collect(self.report(), bufs, cap, 0, 0, 0)

    def check_divergence(self, dt: DeviceTrace, cap: int | None = None, stream=None) -> dict:
        cap = dt.n_blocks if cap is None else cap
        o, bufs = self.alloc_outputs(0, cap, 0, 0)
        ws = self.workspace(self.workspace_size(dt))
        t = dt.c()
        _check(lib().simulee_check_divergence(self.h, ctypes.byref(t), ctypes.c_void_p(o.divergence), cap,
                                              ctypes.c_void_p(self._report.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                              ws.numel(), _stream_ptr(stream)), "simulee_check_divergence")
        self.torch.cuda.synchronize(self.device)
        return self._collect(self.report(), bufs, 0, cap, 0, 0)

    def check_redundant_barriers(self, dt: DeviceTrace, cap: int | None = None, grid_cap: int | None = None,
                                 stream=None) -> dict:
        cap = dt.n_blocks * max(dt.max_barriers, 1) if cap is None else cap
        grid_cap = max(dt.max_barriers, 1) if grid_cap is None else grid_cap
        o, bufs = self.alloc_outputs(0, 0, cap, grid_cap)
        ws = self.workspace(self.workspace_size(dt))
        t = dt.c()
        _check(lib().simulee_check_redundant_barriers(
            self.h, ctypes.byref(t), ctypes.c_void_p(o.redundant), cap, ctypes.c_void_p(o.grid_redundant), grid_cap,
            ctypes.c_void_p(self._report.data_ptr()), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
            _stream_ptr(stream)), "simulee_check_redundant_barriers")
        self.torch.cuda.synchronize(self.device)
        return self._collect(self.report(), bufs, 0, 0, cap, grid_cap)
