"""GPU parity of the warp-aware check (Theorem 1 with its warp conditions) against the oracle.

Traces flagged WARP_AWARE carry a statement word per record; on the device they take the radix-sort
path and each intra-block group is searched pair by pair with the warp predicate. Results must equal
the oracle's byte for byte.
"""
import ctypes

import numpy as np
import pytest

import oracle
import tracegen
from gpu_util import checker, diff, gpu_check
from test_oracle_warp import CASES, _kaldi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", sorted(CASES))
def test_closed_cases(name):
    tr = CASES[name][0]()
    assert diff(gpu_check(tr), oracle.check(tr)) == []


def test_kaldi_same_statement_race():
    tr = _kaldi()
    got = gpu_check(tr)
    assert diff(got, oracle.check(tr)) == []
    assert [(int(r["cls"]), int(r["gtid_first"]), int(r["gtid_second"])) for r in got["races"]] == [(0, 1, 3), (0, 2, 4)]


@pytest.mark.parametrize("chunk", range(2))
def test_random_traces(chunk):
    for seed in range(chunk * 100, chunk * 100 + 100):
        tr = tracegen.random_tiny(seed, block_threads=int(np.random.default_rng(seed).integers(1, 90)))
        tw = tracegen.with_statements(tr, seed=seed, diverge_p=(seed % 4) / 4)
        d = diff(gpu_check(tw), oracle.check(tw))
        assert d == [], f"seed {seed}: {d}"


@pytest.mark.parametrize("nb,bt,ep,dp", [(6, 64, 9, 0.0), (4, 256, 12, 0.1), (2, 1024, 6, 0.5)])
def test_grid_family(nb, bt, ep, dp):
    tr = tracegen.with_statements(tracegen.pattern(nb * 5 + ep, n_blocks=nb, block_threads=bt, n_epochs=ep,
                                                   shared_units=12288, global_units=1 << 20), diverge_p=dp)
    assert diff(gpu_check(tr), oracle.check(tr)) == []


def test_batch_mixes_plain_and_warp_aware():
    from paper_1905_01833_gb300 import simulee
    trs = []
    for i in range(12):
        tr = tracegen.random_tiny(900 + i, block_threads=64)
        trs.append(tracegen.with_statements(tr, seed=i, diverge_p=0.2) if i % 2 else tr)
    trs.append(tracegen.pattern(5, n_blocks=3, block_threads=128, n_epochs=8, shared_units=4096,
                                global_units=1 << 16))
    got = checker().check_batch([simulee.to_device(t) for t in trs])
    for i, tr in enumerate(trs):
        assert diff(got[i], oracle.check(tr)) == [], f"trace {i}"


def test_invalid_flag_combinations():
    import torch
    from paper_1905_01833_gb300 import simulee
    tr = tracegen.with_statements(tracegen.random_tiny(3, n_events=50), diverge_p=0.0)
    dt = simulee.to_device(tr)
    chk = checker()
    ws = chk.workspace(1 << 24)
    o, _ = chk.alloc_outputs(128, tr.n_blocks, tr.n_blocks * 8, 8)
    rep = torch.zeros(simulee.REPORT_BYTES, dtype=torch.uint8, device="cuda")
    for flags, st in ((tracegen.WARP_AWARE | tracegen.UNSORTED, dt.stmt.data_ptr()), (tracegen.WARP_AWARE, None)):
        t = dt.c()
        t.flags = flags
        t.stmt = st
        s = simulee.lib().simulee_check(chk.h, ctypes.byref(t), ctypes.byref(o), ctypes.c_void_p(rep.data_ptr()),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert s == simulee.EINVAL
