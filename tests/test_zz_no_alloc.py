"""The allocation-free entry point (simulee_check_noalloc) against simulee_check.

simulee_check_noalloc serves callers that may not allocate device memory (a
fixed memory plan decided at start-up, or a loop that cannot afford the device
synchronisation of cudaMalloc/cudaFree): it runs the same check in a fixed
scratch array held by the library. This test calls it through the C ABI, twice
in a row on each trace, and requires byte-identical results to the workspace
entry point (integer outputs: the tolerance is zero). It also checks that a
trace needing more scratch than the fixed array is refused up front.

Each result is also compared with the CPU oracle directly. Further cases: calls
on fixed buffers with new trace contents before every call (the context then
replays them as one CUDA graph, which the library's replay diagnostic
confirms), and, in a fresh process, a first call made while the stream is
being captured, which is refused with SIMULEE_EINVAL and leaves the next call
working.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import tracegen

pytestmark = pytest.mark.gpu


def _outputs(simulee, torch, n_events, n_blocks, max_barriers):
    races_cap, div_cap = 2 * n_events + 2, n_blocks
    red_cap, grid_cap = n_blocks * max(max_barriers, 1), max(max_barriers, 1)
    bufs = dict(races=torch.zeros(races_cap * 32, dtype=torch.uint8, device="cuda"),
                divergence=torch.zeros(div_cap * 16, dtype=torch.uint8, device="cuda"),
                redundant=torch.zeros(red_cap * 8, dtype=torch.uint8, device="cuda"),
                grid=torch.zeros(grid_cap * 4, dtype=torch.uint8, device="cuda"))
    o = simulee.Outputs(bufs["races"].data_ptr(), races_cap, bufs["divergence"].data_ptr(), div_cap,
                        bufs["redundant"].data_ptr(), red_cap, bufs["grid"].data_ptr(), grid_cap)
    return o, bufs


def _results(simulee, report, bufs):
    r = simulee.Report.from_buffer_copy(report.cpu().numpy().tobytes())
    sizes = dict(races=32 * r.n_races, divergence=16 * r.n_divergence, redundant=8 * r.n_redundant,
                 grid=4 * r.n_grid_redundant)
    lists = {k: bufs[k][:v].cpu().numpy().tobytes() for k, v in sizes.items()}
    return (r.status, r.bad_kind, r.bad_index, r.n_races, r.n_divergence, r.n_redundant, r.n_grid_redundant), lists


def _traces():
    yield tracegen.c1()
    yield tracegen.pattern(4, n_blocks=4, block_threads=128, n_epochs=9, shared_units=2048, global_units=1 << 14)
    for seed in (3, 17):
        yield tracegen.random_tiny(seed, n_events=300)


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    import torch
    from paper_1905_01833_gb300 import simulee
    lib = simulee.lib()
    chk = simulee.Checker(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for tr in _traces():
        dt = simulee.to_device(tr)
        t = dt.c()
        need = chk.workspace_size(dt)
        assert need <= simulee_noalloc_bytes()

        # reference: the entry point that takes a caller workspace
        o_ref, b_ref = _outputs(simulee, torch, tr.n_events, tr.n_blocks, tr.max_barriers)
        rep_ref = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        assert lib.simulee_check(chk.h, ctypes.byref(t), ctypes.byref(o_ref), ctypes.c_void_p(rep_ref.data_ptr()),
                                 ctypes.c_void_p(ws.data_ptr()), need, stream) == 0
        torch.cuda.synchronize()
        want = _results(simulee, rep_ref, b_ref)
        assert want[0][0] == 0
        assert want == _oracle_results(tr), "the workspace entry point differs from the oracle"

        for call in range(2):
            o, b = _outputs(simulee, torch, tr.n_events, tr.n_blocks, tr.max_barriers)
            rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
            assert lib.simulee_check_noalloc(chk.h, ctypes.byref(t), ctypes.byref(o),
                                             ctypes.c_void_p(rep.data_ptr()), stream) == 0
            torch.cuda.synchronize()
            got = _results(simulee, rep, b)
            assert got[0] == want[0], f"call {call}: report differs"
            for k in want[1]:
                assert got[1][k] == want[1][k], f"call {call}: {k} differs"
    chk.close()


def _oracle_results(tr):
    w = oracle.check(tr)
    head = (w["status"], w["bad_kind"], w["bad_index"], len(w["races"]), len(w["divergence"]), len(w["redundant"]),
            len(w["grid_redundant"]))
    return head, dict(races=w["races"].tobytes(), divergence=w["divergence"].tobytes(),
                      redundant=w["redundant"].tobytes(), grid=w["grid_redundant"].tobytes())


def test_noalloc_on_fixed_buffers_with_new_contents():
    """The same arguments call after call (trace, outputs and report buffers never move) with new
    trace contents before each call: every result equals the oracle's on those contents, and the
    calls after the second are issued as one graph launch."""
    import torch
    from paper_1905_01833_gb300 import simulee
    lib = simulee.lib()
    chk = simulee.Checker(0)
    a = tracegen.pattern(5, n_blocks=3, block_threads=128, n_epochs=9, shared_units=2048, global_units=1 << 14)
    rng = np.random.default_rng(3)
    traces = [a]
    for _ in range(2):   # about 3% of the reads become writes: same dimensions, other results
        ev = a.events.copy()
        flip = (((ev[:, 3] >> 28) & 3) == tracegen.READ) & (rng.random(len(ev)) < 0.03)
        ev[flip, 3] = (ev[flip, 3] & ~np.uint32(3 << 28)) | np.uint32(tracegen.WRITE << 28)
        traces.append(tracegen.Trace(ev, a.barrier_counts, a.n_blocks, a.block_threads, a.shared_units,
                                     a.global_units, a.max_barriers))
    wants = [_oracle_results(t) for t in traces]
    assert len({w[1]["races"] for w in wants}) == 3
    dt = simulee.to_device(a)
    assert chk.workspace_size(dt) <= simulee_noalloc_bytes()
    t = dt.c()
    o, b = _outputs(simulee, torch, a.n_events, a.n_blocks, a.max_barriers)
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    replayed = []
    for k, i in enumerate([0, 1, 2, 0, 2, 1]):
        dt.events.copy_(torch.from_numpy(traces[i].events.view(np.int32).reshape(-1, 4)))
        assert lib.simulee_check_noalloc(chk.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(rep.data_ptr()),
                                         stream) == 0
        torch.cuda.synchronize()
        replayed.append(chk.last_replayed())
        got = _results(simulee, rep, b)
        assert got == wants[i], f"call {k} (contents {i}) differs from the oracle"
    assert replayed[0] is False and all(replayed[2:]), replayed
    chk.close()


_CAPTURE_SCRIPT = r"""
import ctypes, sys
import torch
sys.path.insert(0, sys.argv[1])
import tracegen
from paper_1905_01833_gb300 import simulee
tr = tracegen.random_tiny(5, n_events=200)
dt = simulee.to_device(tr)
chk = simulee.Checker(0)
t = dt.c()
caps = (2 * tr.n_events + 2, tr.n_blocks, tr.n_blocks * max(tr.max_barriers, 1), max(tr.max_barriers, 1))
bufs = [torch.zeros(max(c * w, 16), dtype=torch.uint8, device="cuda") for c, w in zip(caps, (32, 16, 8, 4))]
o = simulee.Outputs(bufs[0].data_ptr(), caps[0], bufs[1].data_ptr(), caps[1], bufs[2].data_ptr(), caps[2],
                    bufs[3].data_ptr(), caps[3])
rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
torch.cuda.synchronize()
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.stream(s):
    g.capture_begin()
    st = simulee.lib().simulee_check_noalloc(chk.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(rep.data_ptr()),
                                             ctypes.c_void_p(s.cuda_stream))
    g.capture_end()
torch.cuda.synchronize()
st2 = simulee.lib().simulee_check_noalloc(chk.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(rep.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
torch.cuda.synchronize()
r = simulee.Report.from_buffer_copy(rep.cpu().numpy().tobytes())
print(st, st2, r.status, r.n_races)
"""


def test_noalloc_first_call_during_capture_is_refused():
    """In a fresh process the first call is made while its stream is being captured: the scratch
    address cannot be looked up then, so the call returns EINVAL and queues nothing; the next call,
    outside the capture, runs the check."""
    from paper_1905_01833_gb300 import simulee
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CAPTURE_SCRIPT, root], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    st, st2, status, n_races = (int(x) for x in out.stdout.split()[-4:])
    assert st == simulee.EINVAL and st2 == simulee.OK and status == 0
    assert n_races == len(oracle.check(tracegen.random_tiny(5, n_events=200))["races"])


def test_noalloc_refuses_traces_larger_than_its_scratch():
    import torch
    from paper_1905_01833_gb300 import simulee
    lib = simulee.lib()
    chk = simulee.Checker(0)
    small = torch.zeros((16, 4), dtype=torch.int32, device="cuda")
    counts = torch.zeros(256, dtype=torch.int32, device="cuda")
    # dimensions only: the size check happens before any device memory is read
    t = simulee.Trace(small.data_ptr(), 50_000_000, counts.data_ptr(), 1, 256, 12288, 0, 7, 0)
    o, _ = _outputs(simulee, torch, 0, 1, 7)
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
    s = lib.simulee_check_noalloc(chk.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(rep.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == simulee.ENOMEM
    chk.close()


def simulee_noalloc_bytes() -> int:
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "simulee.h")
    m = re.search(r"#define SIMULEE_NOALLOC_SCRATCH_BYTES \((\d+)u \* (\d+)u \* (\d+)u\)", open(hdr).read())
    return int(m.group(1)) * int(m.group(2)) * int(m.group(3))
