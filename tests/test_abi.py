"""The C-ABI library builds, loads on a machine without a GPU, and exports
every function that include/thermo.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "thermo.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tp_create", "tp_set_fields", "tp_set_wells", "tp_assemble",
                 "tp_build_preconditioner", "tp_solve", "tp_destroy", "tp_amg_create",
                 "tp_amg_vcycle", "tp_export_level", "tp_apply_preconditioner", "tp_spmv"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header(lib):
    from paper_1902_00095_gb300 import thermo
    assert set(declared_functions()) <= set(thermo.SIGNATURES)


def test_host_only_calls_need_no_gpu(lib):
    from paper_1902_00095_gb300 import thermo
    o = thermo.default_opts()
    assert o.interp == 1 and o.nu_pre == 3 and abs(o.theta - 0.25) < 1e-15
    assert o.nu_post == 4 and o.smoother_S == 2 and o.nu_line == 1 and o.nu_S == 1
    assert o.sell_rows == 0
    assert lib.tp_status_string(-5) == b"AMG setup failed"
    assert lib.tp_status_string(1) == b"not converged"


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_1902_00095_gb300 import thermo
    h = ctypes.c_void_p()
    g = thermo.Grid(0, 4, 4, 10.0, 10.0, 10.0, 9.81)
    f = thermo.Fluid()
    assert lib.tp_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(f), None) == thermo.TP_EINVAL
    assert lib.tp_create(None, ctypes.byref(g), ctypes.byref(f), None) == thermo.TP_EINVAL
    assert lib.tp_solve(None, None, None, None, None, 1e-8, 10, 30, None, 0) == thermo.TP_EINVAL
