"""Repeated identical check calls, replayed as one CUDA graph.

A call whose arguments equal the previous call's is captured (second call)
and replayed (later calls). The graph's kernels read the trace and write the
outputs at run time, so new contents in the same device buffers must give
the new contents' results: every call here is compared with the oracle on
what the buffers held at that moment, with replay on and off.
"""
import ctypes

import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import diff

pytestmark = pytest.mark.gpu


def _variant(tr, seed):
    """The same records with about 2% of the reads turned into writes (same dimensions, still valid)."""
    ev = tr.events.copy()
    rng = np.random.default_rng(seed)
    act = (ev[:, 3] >> 28) & 3
    flip = (act == tracegen.READ) & (rng.random(len(ev)) < 0.02)
    ev[flip, 3] = (ev[flip, 3] & ~np.uint32(3 << 28)) | np.uint32(tracegen.WRITE << 28)
    return tracegen.Trace(ev, tr.barrier_counts, tr.n_blocks, tr.block_threads, tr.shared_units, tr.global_units,
                          tr.max_barriers)


class _FixedCall:
    """simulee_check on fixed device buffers: trace, outputs, report and workspace never move."""

    def __init__(self, chk, tr, races_cap):
        import torch
        from paper_1905_01833_gb300 import simulee
        self.torch, self.simulee, self.chk = torch, simulee, chk
        self.dt = simulee.to_device(tr)
        self.caps = (races_cap, tr.n_blocks, tr.n_blocks * max(tr.max_barriers, 1), max(tr.max_barriers, 1))
        self.outs, self.bufs = chk.alloc_outputs(*self.caps)
        self.ws = torch.empty(chk.workspace_size(self.dt), dtype=torch.uint8, device="cuda:0")
        self.rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda:0")
        self.t = self.dt.c()

    def load(self, tr):
        torch = self.torch
        self.dt.events.copy_(torch.from_numpy(tr.events.view(np.int32).reshape(-1, 4)))
        self.dt.barrier_counts.copy_(torch.from_numpy(tr.barrier_counts.view(np.int32)))

    def __call__(self, outs=None):
        torch, simulee = self.torch, self.simulee
        o = self.outs if outs is None else outs
        st = simulee.lib().simulee_check(self.chk.h, ctypes.byref(self.t), ctypes.byref(o),
                                         ctypes.c_void_p(self.rep.data_ptr()), ctypes.c_void_p(self.ws.data_ptr()),
                                         self.ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == simulee.OK
        torch.cuda.synchronize()
        r = simulee.Report.from_buffer_copy(self.rep.cpu().numpy().tobytes())
        rep = dict(status=r.status, bad_kind=r.bad_kind, bad_index=r.bad_index, n_races=r.n_races,
                   n_divergence=r.n_divergence, n_redundant=r.n_redundant, n_grid_redundant=r.n_grid_redundant)
        return self.chk._collect(rep, self.bufs, *self.caps)


@pytest.mark.parametrize("replay", ["auto", "off"])
@pytest.mark.parametrize("path", [0, 1])
def test_new_contents_in_the_same_buffers(replay, path):
    from paper_1905_01833_gb300 import simulee
    chk = simulee.Checker(0, path=path, graph_replay=simulee.GRAPH_AUTO if replay == "auto" else simulee.GRAPH_OFF)
    a = tracegen.pattern(11, n_blocks=24, block_threads=128, n_epochs=10, shared_units=4096, global_units=1 << 18)
    traces = [a, _variant(a, 1), _variant(a, 2)]
    wants = [oracle.check(t) for t in traces]
    assert len({len(w["races"]) for w in wants}) > 1   # the contents give different results
    call = _FixedCall(chk, a, 2 * a.n_events + 2)
    for i in [0, 1, 2, 0, 2, 1, 1, 0]:
        call.load(traces[i])
        d = diff(call(), wants[i])
        assert d == [], (i, d)
        assert chk.last_launches() > 0
    # another argument (a smaller race list): launched directly, truncated to the canonical prefix
    outs, bufs = chk.alloc_outputs(5, *call.caps[1:])
    call.load(traces[1])
    call(outs)
    got = np.frombuffer(bufs["races"][:5 * 32].cpu().numpy().tobytes(), dtype=wants[1]["races"].dtype)
    assert got.tobytes() == wants[1]["races"][:5].tobytes()
    call.load(traces[2])
    assert diff(call(), wants[2]) == []
    chk.close()


def test_batch_calls_replayed():
    from paper_1905_01833_gb300 import simulee
    chk = simulee.Checker(0)
    base = [tracegen.random_grouped(40 + i, n_events=3000) for i in range(3)]
    var = [_variant(t, 7) for t in base]
    dts = [simulee.to_device(t) for t in base]
    for rnd in range(4):
        src = base if rnd % 2 == 0 else var
        for dt, t in zip(dts, src):
            dt.events.copy_(simulee.to_device(t).events)
        got = chk.check_batch(dts)
        for i, t in enumerate(src):
            assert diff(got[i], oracle.check(t)) == [], (rnd, i)
    chk.close()


def test_single_output_entry_points_replayed():
    """simulee_check_races / _divergence / _redundant_barriers called again and again on fixed buffers
    (each call's arguments equal the previous call's, so the second captures and the rest replay),
    with new trace contents before every call."""
    import torch
    from paper_1905_01833_gb300 import simulee
    L = simulee.lib()
    chk = simulee.Checker(0)
    a = tracegen.pattern(23, n_blocks=12, block_threads=128, n_epochs=10, shared_units=4096, global_units=1 << 18)
    traces = [a, _variant(a, 3), _variant(a, 4)]
    wants = [oracle.check(t) for t in traces]
    assert len({w["races"].tobytes() for w in wants}) == 3 and len({w["redundant"].tobytes() for w in wants}) == 3
    dt = simulee.to_device(a)
    t = dt.c()
    ws = torch.empty(chk.workspace_size(dt), dtype=torch.uint8, device="cuda:0")
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda:0")
    rcap, dcap, bcap, gcap = 2 * a.n_events + 2, a.n_blocks, a.n_blocks * max(a.max_barriers, 1), max(a.max_barriers, 1)
    races = torch.empty(rcap * 32, dtype=torch.uint8, device="cuda:0")
    divs = torch.empty(dcap * 16, dtype=torch.uint8, device="cuda:0")
    bars = torch.empty(bcap * 8, dtype=torch.uint8, device="cuda:0")
    grid = torch.empty(gcap * 4, dtype=torch.uint8, device="cuda:0")
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    wsp, repp = ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(rep.data_ptr())

    def report():
        torch.cuda.synchronize()
        r = simulee.Report.from_buffer_copy(rep.cpu().numpy().tobytes())
        assert r.status == 0
        return r

    def take(buf, n, dtype):
        return np.frombuffer(buf[: n * dtype.itemsize].cpu().numpy().tobytes(), dtype=dtype)

    for name in ("races", "divergence", "redundant"):
        for i in [0, 1, 2, 0, 1, 2]:
            dt.events.copy_(torch.from_numpy(traces[i].events.view(np.int32).reshape(-1, 4)))
            w = wants[i]
            if name == "races":
                assert L.simulee_check_races(chk.h, ctypes.byref(t), ctypes.c_void_p(races.data_ptr()), rcap, repp,
                                             wsp, ws.numel(), sp) == simulee.OK
                r = report()
                assert take(races, r.n_races, simulee.RACE_DTYPE).tobytes() == w["races"].tobytes(), (name, i)
            elif name == "divergence":
                assert L.simulee_check_divergence(chk.h, ctypes.byref(t), ctypes.c_void_p(divs.data_ptr()), dcap,
                                                  repp, wsp, ws.numel(), sp) == simulee.OK
                r = report()
                assert take(divs, r.n_divergence, simulee.DIV_DTYPE).tobytes() == w["divergence"].tobytes(), (name, i)
            else:
                assert L.simulee_check_redundant_barriers(chk.h, ctypes.byref(t), ctypes.c_void_p(bars.data_ptr()),
                                                          bcap, ctypes.c_void_p(grid.data_ptr()), gcap, repp, wsp,
                                                          ws.numel(), sp) == simulee.OK
                r = report()
                assert take(bars, r.n_redundant, simulee.BAR_DTYPE).tobytes() == w["redundant"].tobytes(), (name, i)
                assert take(grid, r.n_grid_redundant, np.dtype("<u4")).tobytes() == w["grid_redundant"].tobytes()
    chk.close()
