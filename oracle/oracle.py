"""ctypes binding of the plain FP64 CPU oracle (wp_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library. It shares no code with the
CUDA path; problems and potentials arrive as plain dictionaries (the schema the
workload module documents) and are marshalled into the oracle's own structs.

Every function follows the paper (arXiv:1306.3247):
  fft / ifft        -- unnormalised DFT of eq. (ft), forward sign -1
  gaussian          -- the normalised packet of Sec. 4.2
  potential_grid    -- V(x,t), the user potential() of Sec. 3.2.3
  step / propagate  -- the split step of eq. (splitop) (VKV or the paper's KVK)
  run               -- Algorithm 1 with observables every nprint steps (Tab. 3)
"""
import ctypes
import os

import numpy as np

from . import build as _build

_SHAPES = {"const": 0, "quad": 1, "linear": 2, "gauss": 3, "morse": 4}
_ENVS = {"none": 0, "gauss": 1, "sin2": 2}
_ORDERS = {"vkv": 0, "kvk": 1}

OBS_FIELDS = ("t", "norm", "x0", "x1", "x2", "p0", "p1", "p2", "xx0", "xx1", "xx2",
              "energy", "ekin", "epot", "autocorr", "step")


class _Problem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("order", ctypes.c_int32),
                ("n", ctypes.c_int64 * 3), ("xmin", ctypes.c_double * 3),
                ("L", ctypes.c_double * 3), ("mass", ctypes.c_double),
                ("hbar", ctypes.c_double), ("dt", ctypes.c_double), ("t0", ctypes.c_double),
                ("vgrid", ctypes.c_void_p)]


class _Term(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("env", ctypes.c_int32),
                ("a", ctypes.c_double * 3), ("c0", ctypes.c_double * 3), ("v", ctypes.c_double * 3),
                ("A0", ctypes.c_double), ("A", ctypes.c_double), ("omega", ctypes.c_double),
                ("phi", ctypes.c_double), ("t0", ctypes.c_double), ("tau", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        c128p = ctypes.c_void_p
        lib.orc_fft1d.argtypes = [c128p, ctypes.c_int64, ctypes.c_int]
        lib.orc_fftnd.argtypes = [c128p, ctypes.c_int32, P(ctypes.c_int64), ctypes.c_int]
        lib.orc_step.argtypes = [P(_Problem), ctypes.c_int32, P(_Term), c128p, ctypes.c_int64]
        lib.orc_propagate.argtypes = [P(_Problem), ctypes.c_int32, P(_Term), c128p,
                                      ctypes.c_int64, ctypes.c_int64]
        lib.orc_run.argtypes = [P(_Problem), ctypes.c_int32, P(_Term), c128p, ctypes.c_int64,
                                ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        lib.orc_run.restype = ctypes.c_int64
        lib.orc_observe.argtypes = [P(_Problem), ctypes.c_int32, P(_Term), c128p, c128p,
                                    ctypes.c_int64, ctypes.c_void_p]
        lib.orc_gaussian.argtypes = [P(_Problem), P(ctypes.c_double), P(ctypes.c_double),
                                     P(ctypes.c_double), c128p]
        lib.orc_potential_grid.argtypes = [P(_Problem), ctypes.c_int32, P(_Term), ctypes.c_double,
                                           ctypes.c_void_p]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().orc_num_threads()


def _problem(pb: dict) -> _Problem:
    p = _Problem()
    p.ndim = int(pb["ndim"])
    p.order = _ORDERS[pb.get("order", "vkv")]
    n = list(pb["n"]) + [1] * (3 - len(pb["n"]))
    xmin = list(pb["xmin"]) + [0.0] * (3 - len(pb["xmin"]))
    L = list(pb["L"]) + [1.0] * (3 - len(pb["L"]))
    for d in range(3):
        p.n[d] = int(n[d])
        p.xmin[d] = float(xmin[d])
        p.L[d] = float(L[d])
    p.mass = float(pb.get("mass", 1.0))
    p.hbar = float(pb.get("hbar", 1.0))
    p.dt = float(pb["dt"])
    p.t0 = float(pb.get("t0", 0.0))
    vg = pb.get("vgrid")
    if vg is not None:
        arr = np.ascontiguousarray(np.asarray(vg, dtype=np.float64).reshape(_shape(pb)))
        p._vgrid_keep = arr  # the array lives as long as the struct
        p.vgrid = arr.ctypes.data
    return p


def _terms(terms):
    arr = (_Term * max(1, len(terms)))()
    for i, tm in enumerate(terms):
        t = arr[i]
        t.shape = _SHAPES[tm["shape"]]
        for d in range(3):
            t.a[d] = float((list(tm.get("a", [])) + [0.0] * 3)[d])
            t.c0[d] = float((list(tm.get("c0", [])) + [0.0] * 3)[d])
            t.v[d] = float((list(tm.get("v", [])) + [0.0] * 3)[d])
        cf = tm.get("coef", {})
        t.env = _ENVS[cf.get("env", "none")]
        t.A0 = float(cf.get("A0", 0.0))
        t.A = float(cf.get("A", 0.0))
        t.omega = float(cf.get("omega", 0.0))
        t.phi = float(cf.get("phi", 0.0))
        t.t0 = float(cf.get("t0", 0.0))
        t.tau = float(cf.get("tau", 1.0))
    return arr, len(terms)


def _shape(pb):
    return tuple(int(x) for x in pb["n"][: int(pb["ndim"])])


def _c128(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a.copy()


def fft(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised multi-dimensional DFT, sign -1 forward, +1 inverse."""
    a = _c128(a)
    n = (ctypes.c_int64 * 3)(*(list(a.shape) + [1] * (3 - a.ndim)))
    _load().orc_fftnd(a.ctypes.data, a.ndim, n, int(sign))
    return a


def gaussian(pb: dict, x0, p0, sigma) -> np.ndarray:
    p = _problem(pb)
    d3 = lambda v: (ctypes.c_double * 3)(*(list(v) + [0.0] * (3 - len(v))))
    sig = list(sigma) + [1.0] * (3 - len(sigma))
    out = np.zeros(_shape(pb), dtype=np.complex128)
    _load().orc_gaussian(ctypes.byref(p), d3(x0), d3(p0), (ctypes.c_double * 3)(*sig), out.ctypes.data)
    return out


def potential_grid(pb: dict, terms, t: float) -> np.ndarray:
    p = _problem(pb)
    arr, nt = _terms(terms)
    out = np.zeros(_shape(pb), dtype=np.float64)
    _load().orc_potential_grid(ctypes.byref(p), nt, arr, float(t), out.ctypes.data)
    return out


def step(pb: dict, terms, psi: np.ndarray, s: int = 0) -> np.ndarray:
    p = _problem(pb)
    arr, nt = _terms(terms)
    psi = _c128(psi, _shape(pb))
    _load().orc_step(ctypes.byref(p), nt, arr, psi.ctypes.data, int(s))
    return psi


def propagate(pb: dict, terms, psi: np.ndarray, nt: int, s0: int = 0) -> np.ndarray:
    p = _problem(pb)
    arr, n = _terms(terms)
    psi = _c128(psi, _shape(pb))
    _load().orc_propagate(ctypes.byref(p), n, arr, psi.ctypes.data, int(s0), int(nt))
    return psi


def observe(pb: dict, terms, psi: np.ndarray, psi0=None, s: int = 0) -> np.ndarray:
    p = _problem(pb)
    arr, n = _terms(terms)
    psi = _c128(psi, _shape(pb))
    rec = np.zeros(16, dtype=np.float64)
    p0 = None
    if psi0 is not None:
        p0 = _c128(psi0, _shape(pb))
    _load().orc_observe(ctypes.byref(p), n, arr, psi.ctypes.data,
                        p0.ctypes.data if p0 is not None else None, int(s), rec.ctypes.data)
    return rec


def run(pb: dict, terms, psi: np.ndarray, nt: int, nprint: int, s0: int = 0):
    """Algorithm 1: returns (final psi, observables array [nobs, 16])."""
    p = _problem(pb)
    arr, n = _terms(terms)
    psi = _c128(psi, _shape(pb))
    if nprint <= 0 or nprint > nt:
        raise ValueError("nprint must satisfy 0 < nprint <= nt")
    obs = np.zeros((1 + nt // nprint, 16), dtype=np.float64)
    k = _load().orc_run(ctypes.byref(p), n, arr, psi.ctypes.data, int(s0), int(nt), int(nprint),
                        obs.ctypes.data)
    return psi, obs[:k]
