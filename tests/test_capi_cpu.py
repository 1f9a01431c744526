"""The C-ABI library builds, loads and exports every entry point of include/dgt.h (no GPU)."""
import ctypes
import os
import subprocess

import pytest

from paper_1307_4569_gb300 import _capi as K
from paper_1307_4569_gb300 import build as B


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    names = K.header_functions()
    for required in ("dgt_plan_create", "dgt_exec", "idgt_exec", "dgt_window_dual", "dgt_window_tight",
                     "dgt_plan_destroy", "dgt_workspace_bytes", "dgt_exec_ws", "idgt_exec_ws"):
        assert required in names
    # every declared function has a ctypes signature in the binding
    assert set(names) <= set(K.SIGNATURES), set(names) - set(K.SIGNATURES)


def test_library_exports_every_header_symbol(libpath):
    assert os.path.exists(libpath)
    h = ctypes.CDLL(libpath)
    for name in K.header_functions():
        assert hasattr(h, name), name


def test_binding_loads_and_reports_errors(libpath):
    lib = K.lib()
    assert lib.dgt_strerror(K.DGT_ERR_LENGTH) == b"DGT_ERR_LENGTH"
    assert lib.dgt_strerror(99) == b"DGT_ERR_UNKNOWN"
    with pytest.raises(K.DGTError):
        K.check(K.DGT_ERR_ARG)


def test_release_build_reports_no_guard_checks(libpath):
    # the guard-zone entry points exist in the release build and say that nothing is checked
    lib = K.lib()
    assert lib.dgt_debug_build() == 0
    v, off, name = ctypes.c_ulonglong(5), ctypes.c_longlong(0), ctypes.create_string_buffer(16)
    assert lib.dgt_debug_status(ctypes.byref(v), ctypes.byref(off), name, 16) == K.DGT_ERR_UNSUPPORTED
    assert v.value == 0 and off.value == -1 and name.value == b""
    assert lib.dgt_debug_touch_guard(None) == K.DGT_ERR_ARG


def test_debug_guard_code_compiles(tmp_path):
    # the DGT_DEBUG-only translation unit (zone registry, check kernel, status) cross-compiles
    cmd = [B._nvcc(), "-c", os.path.join(B.CSRC, "debug.cu"), "-o", str(tmp_path / "debug.o"), "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-I", os.path.join(B.ROOT, "include"), "-I", B.CSRC, "-DDGT_DEBUG"] + B.ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_build_is_incremental(libpath):
    assert B.up_to_date()


def test_wait_limit_hook_sets_queries_and_restores(libpath):
    # host-side state only: the limit later launches pass to their bounded waits
    lib = K.lib()
    default = lib.dgt_wait_limit(-1)
    assert default == 2000000000
    assert lib.dgt_wait_limit(12345) == default
    assert lib.dgt_wait_limit(-1) == 12345
    assert lib.dgt_wait_limit(0) == 12345
    assert lib.dgt_wait_limit(default) == 0
    assert lib.dgt_wait_limit(-1) == default


def test_chirp_table_cap_sets_queries_and_restores(libpath):
    # host-side state only: the cap plans created later apply to their chirp tables
    lib = K.lib()
    default = lib.dgt_chirp_table_cap(-1)
    assert default == 1 << 30
    assert lib.dgt_chirp_table_cap(0) == default
    assert lib.dgt_chirp_table_cap(-1) == 0
    assert lib.dgt_chirp_table_cap(default) == 0
    assert lib.dgt_chirp_table_cap(-1) == default
