"""The C-ABI library loads and exports every entry point include/spmv.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "spmv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spmv_\w+)\s*\(", text)) - {"spmv_handle"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["spmv_create_coo", "spmv_convert", "spmv_mul", "spmv_mul_batch", "spmv_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2502_19284_gb300 as sp
    lib = ctypes.CDLL(sp.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", sp.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (spmv_\w+)", out))
    assert set(declared_functions()) <= exported


def test_status_strings_and_argument_checks_without_gpu():
    import paper_2502_19284_gb300 as sp
    lib = sp._lib
    assert lib.spmv_status_string(sp.SPMV_ERR_INDEX_RANGE) == b"SPMV_ERR_INDEX_RANGE"
    out = ctypes.c_void_p()
    # argument checks happen before any device call
    assert lib.spmv_create_coo(-1, 4, 0, None, None, None, sp.SPMV_F64, 0, None, ctypes.byref(out)) == sp.SPMV_ERR_INVALID_ARG
    assert b"negative" in lib.spmv_last_error()
    assert lib.spmv_create_coo(4, 4, 1 << 31, None, None, None, sp.SPMV_F64, 0, None, ctypes.byref(out)) == sp.SPMV_ERR_UNSUPPORTED
    assert lib.spmv_create_coo(4, 4, 2, None, None, None, sp.SPMV_F64, 0, None, ctypes.byref(out)) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create_coo(4, 4, 0, None, None, None, 7, 0, None, ctypes.byref(out)) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_create_coo(4, 4, 0, None, None, None, sp.SPMV_F64, 0, None, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_convert(None, 0, None, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_mul(None, None, None, 0, 0, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_wait(None, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_mul_batch(1, None, 1, None, None, 0, 0, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_destroy(None) == sp.SPMV_OK
    # serving: option limits are checked before any device call
    out = ctypes.c_void_p()
    for o in [(0, 4, 8), (1 << 30, 0, 8), (1 << 30, 65, 8), (1 << 30, 4, 0), (1 << 30, 4, 2000)]:
        opts = sp.spmv_server_opts(*o)
        assert lib.spmv_server_create(ctypes.byref(opts), ctypes.byref(out)) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_server_add(None, None, None) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_server_destroy(None) == sp.SPMV_OK
    # bounded-wait hook: poll counts outside [1, 2^22] are refused before any device call
    word = ctypes.c_uint32(0)
    for polls in (0, -5, (1 << 22) + 1):
        assert lib.spmv_test_wait_timeout(polls, ctypes.byref(word)) == sp.SPMV_ERR_INVALID_ARG
    assert lib.spmv_test_wait_timeout(10, None) == sp.SPMV_ERR_INVALID_ARG


def test_server_struct_layouts_match_header():
    import paper_2502_19284_gb300 as sp
    assert ctypes.sizeof(sp.spmv_request) == 48 and sp.spmv_request.damping.offset == 24
    assert sp.spmv_request.x.offset == 32 and sp.spmv_request.y.offset == 40
    assert ctypes.sizeof(sp.spmv_server_opts) == 16 and ctypes.sizeof(sp.spmv_server_stats_t) == 64


def test_package_fails_loudly_without_library(tmp_path):
    """Importing the binding with the library absent raises (no CPU fallback)."""
    import shutil
    import sys
    pkg = tmp_path / "paper_2502_19284_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2502_19284_gb300"), pkg,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    code = "import paper_2502_19284_gb300"
    r = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0 and "libspmv.so not built" in r.stderr
