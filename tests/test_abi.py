"""The C ABI library loads and exports every entry point include/vof.h
declares (no compute call: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vof():
    from paper_2407_07463_gb300 import build, vof

    build.build()
    vof.lib()
    return vof


def declared():
    hdr = open(os.path.join(ROOT, "include", "vof.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(vof_[a-z_0-9]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(vof):
    names = declared()
    assert len(names) >= 15
    lib = vof.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing
    assert set(names) == set(vof.EXPORTS)


def test_config_and_workspace_validation(vof):
    cfg = vof.make_config(48, 32, 16, k_capacity=4, k_active=2)
    assert vof.vof_workspace_size(cfg) > 0
    bad = vof.make_config(48, 32, 16, k_capacity=4, k_active=5)
    assert vof.vof_workspace_size(bad) == 0
    bad = vof.make_config(0, 32, 16)
    assert vof.vof_workspace_size(bad) == 0
    bad = vof.make_config(8, 8, 8, connectivity=7)
    assert vof.vof_workspace_size(bad) == 0
    assert vof.lib().vof_status_string(-5) == b"CFL number above 1/2"


def test_init_rejects_null_buffers(vof):
    import ctypes as C
    cfg = vof.make_config(8, 8, 8)
    h = C.c_void_p()
    st = vof.lib().vof_init(C.byref(cfg), None, None, None, 0, None, C.byref(h))
    assert st == -1 and not h.value
