"""Host-side checks that need no GPU: the C-ABI library loads and exports every symbol
declared in include/folty.h; the binding mirrors the header's structs; calls that fail
argument checks before touching the device report the documented status."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "folty.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(folty_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def F():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_17215_gb300 as F
    return F


def test_library_exports_every_declared_symbol(F):
    declared = _declared()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (folty_[a-z_]+)\b", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert sorted(F.EXPORTED) == declared
    for s in declared:
        assert hasattr(F.lib, s)


def _c_struct_sizes():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "folty.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(folty_query_params), sizeof(folty_result),
         sizeof(folty_graph_info), sizeof(folty_traffic_model), sizeof(folty_allocator));
  printf("%zu %zu %zu\n", offsetof(folty_result, n_cert_edges), offsetof(folty_graph_info, triangles),
         offsetof(folty_graph_info, device_bytes));
  return 0;
}'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    return [int(x) for x in lines[0].split()], [int(x) for x in lines[1].split()]


def test_binding_structs_match_header(F):
    sizes, offs = _c_struct_sizes()
    assert sizes == [ctypes.sizeof(F.folty_query_params), ctypes.sizeof(F.folty_result),
                     ctypes.sizeof(F.folty_graph_info), ctypes.sizeof(F.folty_traffic_model),
                     ctypes.sizeof(F.folty_allocator)]
    assert offs == [F.folty_result.n_cert_edges.offset, F.folty_graph_info.triangles.offset,
                    F.folty_graph_info.device_bytes.offset]


def test_argument_errors_before_device_work(F):
    out = ctypes.c_void_p()
    src = np.zeros(1, np.int32)
    t = np.zeros(1, np.int64)
    assert F.lib.folty_load_temporal_graph(-1, 1, src.ctypes.data, src.ctypes.data, t.ctypes.data,
                                           None, None, ctypes.byref(out)) == F.FOLTY_EINVAL
    assert "n outside" in F.folty_last_error()
    assert F.lib.folty_load_temporal_graph(4, 1, None, None, None, None, None,
                                           ctypes.byref(out)) == F.FOLTY_EINVAL
    assert F.lib.folty_load_temporal_graph(4, 1 << 31, src.ctypes.data, src.ctypes.data,
                                           t.ctypes.data, None, None, ctypes.byref(out)) == F.FOLTY_EINVAL
    assert out.value is None
    assert F.lib.folty_preprocess(None, None) == F.FOLTY_EINVAL
    info = F.folty_graph_info()
    assert F.lib.folty_graph_get_info(None, ctypes.byref(info)) == F.FOLTY_EINVAL
    F.lib.folty_free(None)  # no-op


def test_free_ignores_foreign_and_freed_results(F):
    r = F.folty_result()
    F.lib.folty_free(ctypes.byref(r))  # tag 0: ignored
    blob = (ctypes.c_uint64 * 4)(1, 2, 3, 4)
    F.lib.folty_free(blob)  # unknown tag: ignored
