"""The allocation-free entry point (simulee_check_noalloc) against simulee_check.

simulee_check_noalloc serves callers that may not allocate device memory (a
fixed memory plan decided at start-up, or a loop that cannot afford the device
synchronisation of cudaMalloc/cudaFree): it runs the same check in a fixed
scratch array held by the library. This test calls it through the C ABI, twice
in a row on each trace, and requires byte-identical results to the workspace
entry point (integer outputs: the tolerance is zero). It also checks that a
trace needing more scratch than the fixed array is refused up front.

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

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
