"""The C-ABI library builds, loads, and exports every entry point that
include/*.h declares (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(spmspv_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("spmspv_create_csc", "spmspv_run", "spmspv_destroy", "spmspv_last_error",
              "spmspv_device_status"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1610_07902_gb300 import builder as build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, "declared but not exported: %s" % missing


def test_last_error_is_callable_without_gpu():
    from paper_1610_07902_gb300 import builder as build
    lib = ctypes.CDLL(build.build())
    lib.spmspv_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.spmspv_last_error(), bytes)
    # argument checks run on the host before any CUDA call
    lib.spmspv_create_csc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]
    assert lib.spmspv_create_csc(None, 1, 1, 0, None, None, None, 0, 0) == 1  # SPMSPV_ERR_ARG
