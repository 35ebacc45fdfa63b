"""The C-ABI library loads without a GPU and exports every declared entry point."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")) + glob.glob(os.path.join(ROOT, "include", "*.cuh")):
        text = open(h).read()
        # only the extern "C" prototypes: "<type> hr_name(" at line start, ending in ");"
        for m in re.finditer(r"^(?:hr_status|const char\*|void)\s+(hr_\w+)\s*\([^;{]*\);", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2401_04701_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_declarations_found():
    names = declared_functions()
    for must in ("hr_init", "hr_check_trace", "hr_sync", "hr_report", "hr_destroy", "hr_status_str",
                 "hr_device_view"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.hr_status_str.restype = ctypes.c_char_p
    lib.hr_status_str.argtypes = [ctypes.c_int]
    assert lib.hr_status_str(0) == b"ok"
    assert b"range" in lib.hr_status_str(5)
    lib.hr_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hr_version()
    # argument checks happen before any CUDA call
    lib.hr_init.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p]
    assert lib.hr_init(None, None, 0, 1, None) == 1
    out = ctypes.c_void_p()
    assert lib.hr_init(ctypes.byref(out), None, 1, 1, None) == 1
    lib.hr_destroy.argtypes = [ctypes.c_void_p]
    assert lib.hr_destroy(None) == 1


@pytest.mark.parametrize("bad", [dict(shadow_bytes=3), dict(shadow_bytes=8, tid_bits=16),
                                 dict(shadow_bytes=4, tid_bits=3), dict(shadow_bytes=4, tid_bits=23),
                                 dict(shadow_bytes=4, tid_bits=8, block_dim=512), dict(reserved=1)])
def test_init_rejects_bad_shadow_packing(lib, bad):
    """A compact region needs 4 <= tid_bits <= 22 and block_dim <= 2^tid_bits; an
    8-byte region takes no tid width (checked before any CUDA call)."""
    from paper_2401_04701_gb300 import hirace
    arr = (hirace.HrRegionDesc * 1)()
    arr[0].n_words = 64
    arr[0].block_dim = bad.get("block_dim", 256)
    arr[0].warp_size = 32
    arr[0].shadow_bytes = bad.get("shadow_bytes", 0)
    arr[0].tid_bits = bad.get("tid_bits", 0)
    arr[0].reserved = bad.get("reserved", 0)
    lib.hr_init.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.hr_init(ctypes.byref(out), arr, 1, 1024, None) == 1
    assert not out.value
