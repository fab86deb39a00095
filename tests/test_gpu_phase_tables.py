"""The complex64 tables' potential phase factors exp(-i A tau/hbar) (Sec. 2.1, eq.
(splitop)): cosine and sine as float-float pairs with FP64 only in the reduction of the
argument modulo pi/2, checked through the library's probe against the FP64 sincos of the
same argument. The bound is the precision of a table record (high + low FP32 parts, about
48 significant bits)."""
import ctypes
import math

import pytest

from paper_1306_3247_gb300 import wavepacket as WPK

pytestmark = pytest.mark.gpu


def phase_error(n, amax):
    lib = WPK.load_library()
    lib.wp_probe_phase_ff.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.wp_probe_phase_ff.restype = ctypes.c_int
    out = ctypes.c_double(-1.0)
    st = lib.wp_probe_phase_ff(n, amax, None, ctypes.byref(out))
    assert st == WPK.WP_OK, st
    return out.value


@pytest.mark.parametrize("amax", [math.pi / 4, 10.0, 1000.0, 1.0e5])
def test_float_float_phase_matches_fp64_sincos(amax):
    # 2^20 arguments over [-amax, amax]: every quadrant, and arguments near the multiples
    # of pi/2 where the reduced argument is small
    err = phase_error(1 << 20, amax)
    print(f"amax {amax:g}: largest |cos|, |sin| error {err:.3e}")
    assert 0.0 <= err < 2.0 ** -45


def test_probe_rejects_bad_arguments():
    lib = WPK.load_library()
    lib.wp_probe_phase_ff.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.wp_probe_phase_ff.restype = ctypes.c_int
    out = ctypes.c_double(0.0)
    assert lib.wp_probe_phase_ff(0, 1.0, None, ctypes.byref(out)) == WPK.WP_EINVAL
    assert lib.wp_probe_phase_ff(16, -1.0, None, ctypes.byref(out)) == WPK.WP_EINVAL
    assert lib.wp_probe_phase_ff(16, 1.0, None, None) == WPK.WP_EINVAL
