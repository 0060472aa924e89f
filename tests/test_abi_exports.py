"""CPU: the C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/gbx.h declares; the binding's error strings come from it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgbx():
    from paper_2309_07337_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    src = open(os.path.join(ROOT, "include", "gbx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbx_\w+)\s*\(", src)))


def test_header_declares_the_mpi_shaped_calls():
    names = declared()
    for n in ("gbx_comm_create", "gbx_dist_graph_create_adjacent", "gbx_neighbor_alltoallv_init",
              "gbx_start", "gbx_wait", "gbx_startall", "gbx_backward_init", "gbx_request_free"):
        assert n in names


def test_every_declared_symbol_is_exported(libgbx):
    missing = [n for n in declared() if not hasattr(libgbx, n)]
    assert not missing, missing


def test_error_strings_and_version(libgbx):
    libgbx.gbx_error_string.restype = ctypes.c_char_p
    libgbx.gbx_error_string.argtypes = [ctypes.c_int]
    assert libgbx.gbx_error_string(0) == b"success"
    assert b"truncate" in libgbx.gbx_error_string(3).lower() or b"mismatch" in libgbx.gbx_error_string(3)
    assert libgbx.gbx_version() >= 100


def test_host_side_argument_checks(libgbx):
    """Calls that fail before touching the device return GBX_ERR_ARG on any machine."""
    import paper_2309_07337_gb300 as g
    L = g.lib()
    h = ctypes.c_void_p()
    assert L.gbx_comm_create(0, 1, ctypes.byref(h)) == g.ERR_ARG
    assert L.gbx_comm_create(4, 0, ctypes.byref(h)) == g.ERR_ARG
    assert L.gbx_comm_create(4, 2, ctypes.byref(h)) == g.SUCCESS
    r = ctypes.c_void_p()
    assert L.gbx_dist_graph_create_adjacent(h, -1, None, None, None, 0, None, None, None, None, 0,
                                            None, ctypes.byref(r)) == g.ERR_ARG
    assert L.gbx_start(None) == g.ERR_ARG and L.gbx_wait(None) == g.ERR_ARG
    assert L.gbx_startall(0, None) == g.ERR_ARG
    assert L.gbx_comm_free(ctypes.byref(h)) == g.SUCCESS and not h.value


def test_oracle_and_library_error_codes_agree():
    import oracle
    import paper_2309_07337_gb300 as g
    for name in ("ERR_ARG", "ERR_RANK", "ERR_TRUNCATE", "ERR_INDEX", "ERR_DUP", "ERR_GIDX",
                 "ERR_NOMEM", "ERR_OVERLAP"):
        assert getattr(oracle, name) == getattr(g, name)
    hdr = open(os.path.join(ROOT, "include", "gbx.h")).read()
    for name, val in re.findall(r"#define GBX_(ERR_\w+)\s+(\d+)", hdr):
        assert getattr(g, name) == int(val), name
