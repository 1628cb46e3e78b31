"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/hsma.h.

No compute call is made here (this runs without a GPU)."""
import os
import re

from paper_1907_01724_gb300 import _native

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hsma.h")


def declared_functions():
    text = open(HEADER).read()
    return set(re.findall(r"^HSMA_API\s+[\w\s\*]+?\b(hsma_\w+)\s*\(", text, flags=re.M))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("hsma_create", "hsma_build_sources", "hsma_potential", "hsma_energy", "hsma_delta_energy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    exported = _native.exported_symbols()
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_reports_version():
    lib = _native.load()
    assert b"sm_103a" in lib.hsma_version()
    for name in declared_functions():
        assert hasattr(lib, name)


def test_default_params_without_gpu():
    import ctypes
    lib = _native.load()
    p = _native.HsmaParams()
    assert lib.hsma_default_params(ctypes.byref(p)) == 0
    assert p.p == 20 and p.M == 1000 and abs(p.tau - 0.1) < 1e-15 and abs(p.dy_rel - 1e-5) < 1e-20
    assert lib.hsma_default_params(None) == -1


def test_built_for_sm103a_only():
    assert _native.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_server_entry_points_reject_null_without_gpu():
    import ctypes
    lib = _native.load()
    cnt = ctypes.c_int()
    assert lib.hsma_server_start(None) == -1
    assert lib.hsma_server_submit(None, None, None) == -1
    assert lib.hsma_server_poll(None, None, 0, 0.0, ctypes.byref(cnt)) == -1
    assert lib.hsma_server_stop(None, 1) == -1
