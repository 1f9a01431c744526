"""The C-ABI library builds, loads and exports every entry point of include/dgt.h (no GPU)."""
import ctypes
import os

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
