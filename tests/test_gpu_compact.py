"""Compact workspaces: the check lays its record streams and race staging out in
the workspace it is given. With simulee_compact_workspace_size bytes, traces in
simulator order (the hash path) give exactly the oracle's results; a call that
meets more sort-path records or races than the workspace holds reports ENOMEM
(and the full workspace then gives the oracle's results); a workspace below the
compact size is refused on the host; the server re-checks such jobs with the
full workspace."""
import ctypes

import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import checker, diff

pytestmark = pytest.mark.gpu


def _racy_trace(n_blocks=1024, bt=1024):
    """Every shared unit t of every block written by threads t and t+1 (one epoch): n/2 WW races,
    far more than a compact workspace stages."""
    b = np.repeat(np.arange(n_blocks, dtype=np.int64), 2 * bt)
    k = np.tile(np.arange(2 * bt, dtype=np.int64), n_blocks)
    unit = k % bt
    tid = np.where(k < bt, unit, (unit + 1) % bt)
    ev = tracegen.pack(unit, np.arange(len(b)), b, tid, 0, tracegen.WRITE, tracegen.SHARED)
    return tracegen.Trace(ev, np.zeros(n_blocks * bt, dtype=np.uint32), n_blocks, bt, bt, 0, 0)


def test_compact_workspace_grid_family_equals_oracle():
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.pattern(8, n_blocks=96, block_threads=256, n_epochs=32, shared_units=12288, global_units=1 << 20)
    dt = simulee.to_device(tr)
    chk = checker()
    full, comp = chk.workspace_size(dt), chk.compact_workspace_size([dt])
    assert comp * 3 < full, (comp, full)
    assert comp / tr.n_events <= 48, comp / tr.n_events
    got = chk.check(dt, compact=True)
    assert diff(got, oracle.check(tr)) == []


def test_compact_batch_with_sort_path_traces_equals_oracle():
    from paper_1905_01833_gb300 import simulee
    trs = [tracegen.c3_trace(i, 20000 + 3000 * i, (64, 128, 256, 1024)[i % 4], 4 + 7 * i, seed=21) for i in range(8)]
    trs += [tracegen.random_tiny(s, unsorted=True, n_events=400) for s in range(3)]
    trs += [tracegen.with_statements(tracegen.random_grouped(5, n_events=300))]
    pap = tracegen.random_grouped(6, n_events=300)
    pap.flags |= tracegen.PAPER_ORDER
    trs.append(pap)
    got = checker().check_batch([simulee.to_device(t) for t in trs], compact=True)
    for i, t in enumerate(trs):
        assert diff(got[i], oracle.check(t)) == [], f"trace {i}"


def test_overflow_reports_enomem_and_the_full_workspace_is_right():
    from paper_1905_01833_gb300 import simulee
    tr = _racy_trace()
    dt = simulee.to_device(tr)
    chk = checker()
    got = chk.check(dt, compact=True)
    assert got["status"] == simulee.ENOMEM
    assert diff(chk.check(dt), oracle.check(tr)) == []


def test_workspace_below_the_compact_size_is_refused():
    import torch
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.pattern(9, n_blocks=8, block_threads=256, n_epochs=8, shared_units=12288, global_units=1 << 18)
    dt = simulee.to_device(tr)
    chk = checker()
    comp = chk.compact_workspace_size([dt])
    outs, _ = chk.alloc_outputs(2 * tr.n_events + 2, tr.n_blocks, tr.n_blocks * tr.max_barriers, tr.max_barriers)
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda:0")
    ws = torch.empty(comp, dtype=torch.uint8, device="cuda:0")
    t = dt.c()
    small = comp // 4
    s = simulee.lib().simulee_check(chk.h, ctypes.byref(t), ctypes.byref(outs), ctypes.c_void_p(rep.data_ptr()),
                                    ctypes.c_void_p(ws.data_ptr()), small,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == simulee.ENOMEM


def test_server_rechecks_jobs_that_overflow_a_compact_workspace():
    from paper_1905_01833_gb300 import serve, simulee
    trs = [_racy_trace(), tracegen.pattern(3, n_blocks=16, block_threads=256, n_epochs=12, shared_units=12288,
                                           global_units=1 << 18), tracegen.c1()]
    dts = [simulee.to_device(t) for t in trs]
    jobs = [serve.Job(i, dts[i % 3], 1e-4 * i, races_cap=2 * trs[i % 3].n_events + 2) for i in range(9)]
    stats = serve.Server(0, hbm_budget=16 << 30).run(jobs)
    assert stats["retried"] >= 1, stats
    wants = [oracle.check(t) for t in trs]
    for j in jobs:
        assert diff(j.result, wants[j.jid % 3]) == [], f"job {j.jid}"
