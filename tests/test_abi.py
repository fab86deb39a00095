"""The C-ABI library builds, loads without a GPU and exports every entry point the
public header declares (no compute call is made)."""
import ctypes
import os
import re

from paper_1306_3247_gb300 import build as B

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(wp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("wp_create", "wp_set_potential", "wp_set_state", "wp_init_gaussian", "wp_run", "wp_step",
              "wp_observe", "wp_get_state", "wp_fft", "wp_state_ptr", "wp_destroy", "wp_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_reports_static_metadata_without_gpu():
    lib = ctypes.CDLL(B.build())
    lib.wp_kernel_count.restype = ctypes.c_int
    lib.wp_kernel_name.restype = ctypes.c_char_p
    lib.wp_kernel_name.argtypes = [ctypes.c_int]
    lib.wp_status_string.restype = ctypes.c_char_p
    lib.wp_status_string.argtypes = [ctypes.c_int]
    k = lib.wp_kernel_count()
    assert k >= 5
    assert all(lib.wp_kernel_name(i) for i in range(k))
    assert lib.wp_status_string(0) == b"ok"


def test_autotune_cache_calls_without_gpu():
    lib = ctypes.CDLL(B.build())
    lib.wp_autotune_cache_size.restype = ctypes.c_int64
    lib.wp_autotune_cache_clear.restype = None
    lib.wp_autotune_cache_clear()
    assert lib.wp_autotune_cache_size() == 0
