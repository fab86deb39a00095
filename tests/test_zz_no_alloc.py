"""The allocation-free moments entry point (wp_moments_noalloc), through the C ABI.

It is for callers that cannot allocate device memory; its scratch is a fixed device
array inside the library. Two calls in a row on the same state must agree with the
handle's own observables (wp_observe, which uses allocated scratch) to FP64 rounding,
up to the documented limit of 16,777,216 points (256^3), where every block slot of the
fixed array is in use and the record sits right after the last one.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _lib():
    lib = WPK.load_library()
    lib.wp_moments_noalloc.argtypes = [ctypes.POINTER(WPK.WpProblem), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(WPK.WpObs)]
    lib.wp_moments_noalloc.restype = ctypes.c_int
    lib.wp_moments_noalloc_error.restype = ctypes.c_char_p
    return lib


def _moments(lib, prop, stream=0):
    out = WPK.WpObs()
    st = lib.wp_moments_noalloc(ctypes.byref(prop._pb), ctypes.c_void_p(WPK.wp_state_ptr(prop.h)),
                                ctypes.c_void_p(stream), ctypes.byref(out))
    assert st == WPK.WP_OK, lib.wp_moments_noalloc_error()
    return out


def _check(o, ref, ndim):
    assert abs(o.norm - ref["norm"]) <= RTOL * abs(ref["norm"])
    for d in range(ndim):
        sx = max(abs(ref["x%d" % d]), abs(ref["xx%d" % d]) ** 0.5, 1e-300)
        assert abs(o.x[d] - ref["x%d" % d]) <= RTOL * max(sx, abs(ref["norm"]))
        assert abs(o.x2[d] - ref["xx%d" % d]) <= RTOL * abs(ref["xx%d" % d])


@pytest.mark.parametrize("cfg", [W.config_1d_driven_trap(), W.config_3d_barrier(n=64), W.config_2d_laser_trap(n=256),
                                 W.config_3d_barrier(n=256)],
                         ids=["1d", "3d", "2d", "3d_256_at_the_limit"])
def test_noalloc_moments_match_observe_twice(cfg):
    lib = _lib()
    pb = cfg["problem"]
    with WPK.Propagator(pb, cfg["terms"], "c128") as P:
        P.init_gaussian(**cfg["init"])
        P.step(5)
        ref = P.observe()
        a = _moments(lib, P)
        b = _moments(lib, P)
        _check(a, ref, pb["ndim"])
        _check(b, ref, pb["ndim"])
        assert a.norm == b.norm and list(a.x) == list(b.x)
        # a different state right after: the shared array keeps no stale partial sums
        P.set_state(W.random_state(P.shape, seed=9))
        ref2 = P.observe()
        c = _moments(lib, P)
        _check(c, ref2, pb["ndim"])


def test_noalloc_rejects_oversize_and_null():
    lib = _lib()
    big = WPK.make_problem({"ndim": 3, "n": [512, 512, 128], "xmin": [0, 0, 0], "L": [1, 1, 1], "dt": 0.1})
    out = WPK.WpObs()
    # the size check comes before any device work, so no state is needed
    st = lib.wp_moments_noalloc(ctypes.byref(big), ctypes.c_void_p(1), None, ctypes.byref(out))
    assert st == WPK.WP_EUNSUPPORTED
    assert b"16777216" in lib.wp_moments_noalloc_error()
    st = lib.wp_moments_noalloc(ctypes.byref(big), None, None, ctypes.byref(out))
    assert st == WPK.WP_EINVAL
