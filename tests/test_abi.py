"""The C ABI library loads without a GPU and exports every entry point that
include/simulee.h declares; the Python binding's structures match the header's
layout (checked by compiling a C probe against the header with gcc)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "simulee.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_1905_01833_gb300 import _build
    return _build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(simulee_[a-z_]+)\s*\(", text)))


def test_header_declares_the_check_entry_points():
    names = declared_functions()
    for n in ("simulee_check_races", "simulee_check_divergence", "simulee_check_redundant_barriers",
              "simulee_check", "simulee_check_batch", "simulee_create", "simulee_destroy",
              "simulee_workspace_size", "simulee_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.simulee_status_str.restype = ctypes.c_char_p
    assert lib.simulee_status_str(0) == b"ok"
    assert b"capacity" in lib.simulee_status_str(4)


def test_binding_structs_match_header(tmp_path):
    from paper_1905_01833_gb300 import simulee as S
    probe = tmp_path / "probe.c"
    probe.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "simulee.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(simulee_trace), sizeof(simulee_outputs), sizeof(simulee_report),
         sizeof(simulee_options), sizeof(simulee_race), sizeof(simulee_divergence), sizeof(simulee_barrier),
         sizeof(simulee_fitness));
  printf("%zu %zu %zu %zu\\n", offsetof(simulee_trace, barrier_counts), offsetof(simulee_trace, flags),
         offsetof(simulee_report, n_grid_redundant), offsetof(simulee_race, gtid_second));
  return 0;
}
""")
    exe = str(tmp_path / "probe")
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, str(probe)])
    a, b = subprocess.check_output([exe]).decode().split("\n")[:2]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(S.Trace), ctypes.sizeof(S.Outputs), ctypes.sizeof(S.Report),
                     ctypes.sizeof(S.Options), S.RACE_DTYPE.itemsize, S.DIV_DTYPE.itemsize, S.BAR_DTYPE.itemsize,
                     ctypes.sizeof(S.Fitness)]
    assert offs == [S.Trace.barrier_counts.offset, S.Trace.flags.offset, S.Report.n_grid_redundant.offset,
                    S.RACE_DTYPE.fields["gtid_second"][1]]


def test_oracle_result_layout_matches_binding():
    import oracle
    from paper_1905_01833_gb300 import simulee as S
    assert oracle.RACE_DTYPE == S.RACE_DTYPE and oracle.DIV_DTYPE == S.DIV_DTYPE and oracle.BAR_DTYPE == S.BAR_DTYPE
