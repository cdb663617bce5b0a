"""The C-ABI library builds, loads and exports every symbol include/bcm.h
declares; struct layouts agree with the header; host-side argument checks
answer without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bcm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1507_01490_gb300 import _build, bcm
    _build.build_cuda()
    return bcm


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w ]*[ *]+(bcm_\w+)\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "bcm_topk" in names and "bcm_graph_create" in names
    so = lib.load()
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported
    assert set(lib.EXPORTS) == set(names)


def test_struct_layouts_match_header(lib, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "bcm.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bcm_options), sizeof(bcm_stats),'
                   ' offsetof(bcm_options, wait_limit_ns), offsetof(bcm_stats, kernel_ms), sizeof(bcm_key),'
                   ' offsetof(bcm_key, id), offsetof(bcm_options, cta_table));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(lib.bcm_options), ctypes.sizeof(lib.bcm_stats),
                   lib.bcm_options.wait_limit_ns.offset, lib.bcm_stats.kernel_ms.offset,
                   ctypes.sizeof(lib.bcm_key), lib.bcm_key.id.offset, lib.bcm_options.cta_table.offset]


def test_host_argument_checks(lib):
    so = lib.load()
    key = lib.bcm_key()
    assert so.bcm_topk_threshold(None, ctypes.byref(key)) == lib.BCM_ERR_INVALID
    assert so.bcm_topk_offer(None, ctypes.byref(key)) == lib.BCM_ERR_INVALID
    h = ctypes.c_void_p()
    assert so.bcm_graph_create(None, None, 4, 0, 0, 0, None, 0, ctypes.byref(h)) == lib.BCM_ERR_INVALID
    assert "NULL" in lib.bcm_last_error()
    assert so.bcm_graph_create(None, None, 4, 0, 0, 0, None, 0, None) == lib.BCM_ERR_INVALID
    rp = (ctypes.c_uint64 * 2)(0, 0)
    assert so.bcm_graph_create(rp, None, 1 << 30, 0, 0, 0, None, 0, ctypes.byref(h)) == lib.BCM_ERR_UNSUPPORTED
    ids = (ctypes.c_uint32 * 1)()
    f = (ctypes.c_uint64 * 1)()
    assert so.bcm_topk(None, 1, None, ids, f, ids, None) == lib.BCM_ERR_INVALID
    assert so.bcm_farness_all(None, None, f, ids, None) == lib.BCM_ERR_INVALID
    assert so.bcm_preprocess(None, None, None, None, 0) == lib.BCM_ERR_INVALID
    assert so.bcm_graph_destroy(None) == lib.BCM_OK
    assert so.bcm_workspace_bytes(None, None) == 0
    with pytest.raises(lib.BcmError) as ei:
        lib.bcm_graph_create(None, None, 3, 0, False)
    assert ei.value.status == lib.BCM_ERR_INVALID


def test_binding_refuses_non_contiguous(lib):
    import numpy as np
    a = np.zeros((4, 4), np.uint32)[:, 1]
    with pytest.raises(ValueError):
        lib._ptr(a)
