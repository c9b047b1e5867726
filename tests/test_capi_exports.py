"""The C-ABI library builds, loads without a GPU, and exports every symbol
that include/wmgct.h declares (no compute calls here)."""
import ctypes
import os
import re

import paper_1310_0956_gb300 as wmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(wmg_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_loads_and_exports_declared_symbols():
    lib = wmg.lib()
    names = declared_symbols()
    assert "wmg_plan_create" in names and "wmg_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(wmg.exported_symbols()) >= names


def test_version_and_error_buffer():
    assert wmg.lib().wmg_version() >= 100
    buf = ctypes.create_string_buffer(8)
    assert wmg.lib().wmg_last_error(buf, len(buf)) == 0


def test_invalid_arguments_are_rejected_without_gpu_work():
    geom = wmg.wmg_geom(30, 10, None, 43, 1.0, 0.0)
    opts = wmg.wmg_opts(4, 1, 1, 1.0, 0.0, 2, wmg.CYCLE_SYMMETRIC, wmg.PREC_F64)   # 30 % 8 != 0
    out = ctypes.c_void_p()
    rc = wmg.lib().wmg_plan_create(ctypes.byref(geom), ctypes.byref(opts), None, ctypes.byref(out))
    assert rc == -1 and not out.value
    assert "divisible" in wmg.last_error()
    opts = wmg.wmg_opts(1, 0, 0, 1.0, -1.0, 0, 0, 0)                                 # lambda < 0
    rc = wmg.lib().wmg_plan_create(ctypes.byref(geom), ctypes.byref(opts), None, ctypes.byref(out))
    assert rc == -1


def test_allocator_arguments_are_checked_without_gpu_work():
    # wmg_set_allocator only records the functions: no CUDA call
    alloc = wmg._ALLOC_FN(lambda nbytes, stream, ctx: None)
    try:
        wmg.wmg_set_allocator(alloc, None)
        raise AssertionError("an allocator without its free function was accepted")
    except wmg.WmgError as e:
        assert e.code == wmg.WMG_ERR_INVALID_ARG
    wmg.wmg_set_allocator(None, None)
    assert wmg.WMG_ERR_OOM == -2 and wmg.WMG_ERR_REJECTED == -8
