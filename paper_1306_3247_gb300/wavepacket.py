"""Python binding of the C ABI in include/wavepacket_gpu.h (argument marshalling only).

Every function here forwards to libwavepacket_gpu.so; all arithmetic of the
split-operator step (arXiv:1306.3247, Sec. 2.1) runs in its CUDA kernels. There is
no CPU fallback: if the library is missing or fails to load, importing the handle
raises.

The low-level names match the C ABI (wp_create, wp_set_potential, ...). The
Propagator class wraps one handle and accepts the problem/potential dictionaries
documented in workloads.py.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

WP_OK, WP_EINVAL, WP_EUNSUPPORTED, WP_ENOMEM, WP_ENONFINITE, WP_ETIMEOUT, WP_ECUDA, WP_EBUSY = range(8)
WP_C128, WP_C64, WP_C128_F32X2 = 0, 1, 2
WP_ORDER_VKV, WP_ORDER_KVK = 0, 1
WP_MAX_TERMS = 8
WP_MAX_GAUSS = 2
SHAPES = {"const": 0, "quad": 1, "linear": 2, "gauss": 3, "morse": 4}
ENVS = {"none": 0, "gauss": 1, "sin2": 2}
PRECISIONS = {"c128": WP_C128, "c64": WP_C64, "c128f": WP_C128_F32X2}
ORDERS = {"vkv": WP_ORDER_VKV, "kvk": WP_ORDER_KVK}


class WpProblem(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("precision", ctypes.c_int32), ("order", ctypes.c_int32),
                ("autocorr", ctypes.c_int32), ("n", ctypes.c_int64 * 3), ("xmin", ctypes.c_double * 3),
                ("L", ctypes.c_double * 3), ("mass", ctypes.c_double), ("hbar", ctypes.c_double),
                ("dt", ctypes.c_double), ("t0", ctypes.c_double)]


class WpPotTerm(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("env", ctypes.c_int32), ("a", ctypes.c_double * 3),
                ("c0", ctypes.c_double * 3), ("v", ctypes.c_double * 3), ("A0", ctypes.c_double),
                ("A", ctypes.c_double), ("omega", ctypes.c_double), ("phi", ctypes.c_double),
                ("t0", ctypes.c_double), ("tau", ctypes.c_double)]


class WpPotential(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int32), ("reserved", ctypes.c_int32), ("term", WpPotTerm * WP_MAX_TERMS)]


class WpObs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("norm", ctypes.c_double), ("x", ctypes.c_double * 3),
                ("p", ctypes.c_double * 3), ("x2", ctypes.c_double * 3), ("energy", ctypes.c_double),
                ("ekin", ctypes.c_double), ("epot", ctypes.c_double), ("autocorr", ctypes.c_double),
                ("step", ctypes.c_int64)]


OBS_DTYPE = np.dtype([(n, "<f8") for n in ("t", "norm", "x0", "x1", "x2", "p0", "p1", "p2", "xx0", "xx1", "xx2",
                                            "energy", "ekin", "epot", "autocorr")] + [("step", "<i8")])


class WpSchedule(ctypes.Structure):
    _fields_ = [("tile_log", ctypes.c_int32), ("ept", ctypes.c_int32), ("max_radix_log", ctypes.c_int32),
                ("fixed", ctypes.c_int32)]


RECORD_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class WavepacketError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libwavepacket_gpu.so (building it in-tree first when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    H = vp
    sig = {
        "wp_create": ([P(WpProblem), vp, P(vp)], ctypes.c_int),
        "wp_create_pooled": ([P(WpProblem), vp, vp, P(vp)], ctypes.c_int),
        "wp_set_potential": ([H, P(WpPotential)], ctypes.c_int),
        "wp_set_state": ([H, vp, ctypes.c_int], ctypes.c_int),
        "wp_init_gaussian": ([H, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)], ctypes.c_int),
        "wp_get_state": ([H, vp, ctypes.c_int], ctypes.c_int),
        "wp_step": ([H, ctypes.c_int64], ctypes.c_int),
        "wp_observe": ([H, P(WpObs)], ctypes.c_int),
        "wp_run": ([H, ctypes.c_int64, ctypes.c_int64, vp, P(ctypes.c_int64)], ctypes.c_int),
        "wp_fft": ([H, ctypes.c_int], ctypes.c_int),
        "wp_state_ptr": ([H], vp),
        "wp_get_step_index": ([H], ctypes.c_int64),
        "wp_set_step_index": ([H, ctypes.c_int64], ctypes.c_int),
        "wp_profile_enable": ([H, ctypes.c_int], ctypes.c_int),
        "wp_profile_read": ([H, ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_double)], ctypes.c_int),
        "wp_kernel_count": ([], ctypes.c_int),
        "wp_kernel_name": ([ctypes.c_int], ctypes.c_char_p),
        "wp_launch_count": ([H], ctypes.c_int64),
        "wp_set_potential_grid": ([H, vp, ctypes.c_int], ctypes.c_int),
        "wp_expect_grid": ([H, vp, ctypes.c_int, P(ctypes.c_double)], ctypes.c_int),
        "wp_run_callback": ([H, ctypes.c_int64, ctypes.c_int64, RECORD_FN, vp, P(ctypes.c_int64)], ctypes.c_int),
        "wp_set_potential_source": ([H, ctypes.c_char_p], ctypes.c_int),
        "wp_set_graphs": ([H, ctypes.c_int], ctypes.c_int),
        "wp_get_schedule": ([H, P(WpSchedule)], ctypes.c_int),
        "wp_set_schedule": ([H, P(WpSchedule)], ctypes.c_int),
        "wp_autotune": ([H, ctypes.c_int32, P(WpSchedule), P(ctypes.c_double), P(ctypes.c_int32)], ctypes.c_int),
        "wp_autotune_cache_size": ([], ctypes.c_int64),
        "wp_autotune_cache_clear": ([], None),
        "wp_destroy": ([H], ctypes.c_int),
        "wp_last_error": ([H], ctypes.c_char_p),
        "wp_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "wp_batch_create": ([ctypes.c_int32, vp, P(vp)], ctypes.c_int),
        "wp_batch_add": ([vp, P(WpProblem), P(WpPotential), P(ctypes.c_int64)], ctypes.c_int),
        "wp_batch_handle": ([vp, ctypes.c_int64], vp),
        "wp_batch_size": ([vp], ctypes.c_int64),
        "wp_batch_step": ([vp, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
        "wp_batch_launch_count": ([vp], ctypes.c_int64),
        "wp_batch_destroy": ([vp], ctypes.c_int),
        "wp_batch_last_error": ([vp], ctypes.c_char_p),
        "wp_server_create": ([ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, P(vp)], ctypes.c_int),
        "wp_server_submit": ([vp, ctypes.c_int64, P(WpProblem), P(WpPotential), P(ctypes.c_double),
                              P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int64], ctypes.c_int),
        "wp_server_progress": ([vp, P(ctypes.c_int64), ctypes.c_int64, P(ctypes.c_int64)], ctypes.c_int),
        "wp_server_fetch": ([vp, ctypes.c_int64, vp, P(WpObs), P(ctypes.c_double)], ctypes.c_int),
        "wp_server_pending": ([vp], ctypes.c_int64),
        "wp_server_bytes_in_use": ([vp], ctypes.c_int64),
        "wp_server_running": ([vp], ctypes.c_int32),
        "wp_server_destroy": ([vp], ctypes.c_int),
        "wp_server_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(lib, h, st):
    if st != WP_OK:
        msg = lib.wp_last_error(h).decode(errors="replace") or lib.wp_status_string(st).decode()
        raise WavepacketError(st, msg)


def _vec3(v, fill):
    v = list(v) if v is not None else []
    return (ctypes.c_double * 3)(*[float(x) for x in (v + [fill] * 3)[:3]])


def make_problem(pb: dict, precision="c128", autocorr=False) -> WpProblem:
    p = WpProblem()
    p.ndim = int(pb["ndim"])
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.order = ORDERS[pb.get("order", "vkv")]
    p.autocorr = 1 if autocorr else 0
    n = list(pb["n"]) + [1] * 3
    for d in range(3):
        p.n[d] = int(n[d])
    p.xmin = _vec3(pb["xmin"], 0.0)
    p.L = _vec3(pb["L"], 1.0)
    p.mass = float(pb.get("mass", 1.0))
    p.hbar = float(pb.get("hbar", 1.0))
    p.dt = float(pb["dt"])
    p.t0 = float(pb.get("t0", 0.0))
    return p


def make_potential(terms) -> WpPotential:
    pot = WpPotential()
    if len(terms) > WP_MAX_TERMS:
        raise ValueError(f"at most {WP_MAX_TERMS} potential terms")
    pot.nterms = len(terms)
    for i, tm in enumerate(terms):
        t = pot.term[i]
        t.shape = SHAPES[tm["shape"]]
        t.a = _vec3(tm.get("a"), 0.0)
        t.c0 = _vec3(tm.get("c0"), 0.0)
        t.v = _vec3(tm.get("v"), 0.0)
        cf = tm.get("coef", {})
        t.env = ENVS[cf.get("env", "none")]
        t.A0 = float(cf.get("A0", 0.0))
        t.A = float(cf.get("A", 0.0))
        t.omega = float(cf.get("omega", 0.0))
        t.phi = float(cf.get("phi", 0.0))
        t.t0 = float(cf.get("t0", 0.0))
        t.tau = float(cf.get("tau", 1.0))
    return pot


# ---------------------------------------------------------------- C ABI names
def wp_create(problem: WpProblem, stream=None, mem_pool=None):
    """mem_pool: a cudaMemPool_t (int address) to take the handle's device memory from."""
    lib = load_library()
    h = ctypes.c_void_p()
    if mem_pool:
        st = lib.wp_create_pooled(ctypes.byref(problem), ctypes.c_void_p(stream or 0), ctypes.c_void_p(mem_pool),
                                  ctypes.byref(h))
    else:
        st = lib.wp_create(ctypes.byref(problem), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    _check(lib, None, st)
    return h


def wp_set_potential(h, pot: WpPotential):
    lib = load_library()
    _check(lib, h, lib.wp_set_potential(h, ctypes.byref(pot)))


def wp_set_potential_grid(h, ptr, on_device: bool):
    lib = load_library()
    _check(lib, h, lib.wp_set_potential_grid(h, ctypes.c_void_p(ptr or 0), 1 if on_device else 0))


def wp_set_graphs(h, enable: bool):
    lib = load_library()
    _check(lib, h, lib.wp_set_graphs(h, 1 if enable else 0))


def wp_expect_grid(h, ptr: int, on_device: bool) -> float:
    lib = load_library()
    out = ctypes.c_double(0.0)
    _check(lib, h, lib.wp_expect_grid(h, ctypes.c_void_p(ptr), 1 if on_device else 0, ctypes.byref(out)))
    return out.value


def wp_run_callback(h, nt: int, nprint: int, fn):
    """fn(handle, record) -> truthy to stop; returns the number of records delivered."""
    lib = load_library()
    err = []

    def tramp(hp, rec_ptr, user):
        try:
            rec = _obs_array(rec_ptr, 1)[0]
            return 1 if fn(hp, rec) else 0
        except Exception as e:  # stop the run and re-raise after it returns
            err.append(e)
            return 1

    cb = RECORD_FN(tramp)
    n = ctypes.c_int64(0)
    st = lib.wp_run_callback(h, int(nt), int(nprint), cb, None, ctypes.byref(n))
    if err:
        raise err[0]
    _check(lib, h, st)
    return n.value


def wp_set_potential_source(h, src: str):
    lib = load_library()
    _check(lib, h, lib.wp_set_potential_source(h, src.encode()))


def wp_set_state(h, ptr: int, on_device: bool):
    lib = load_library()
    _check(lib, h, lib.wp_set_state(h, ctypes.c_void_p(ptr), 1 if on_device else 0))


def wp_get_state(h, ptr: int, on_device: bool):
    lib = load_library()
    _check(lib, h, lib.wp_get_state(h, ctypes.c_void_p(ptr), 1 if on_device else 0))


def wp_init_gaussian(h, x0, p0, sigma):
    lib = load_library()
    _check(lib, h, lib.wp_init_gaussian(h, _vec3(x0, 0.0), _vec3(p0, 0.0), _vec3(sigma, 1.0)))


def wp_step(h, nsteps: int):
    lib = load_library()
    _check(lib, h, lib.wp_step(h, int(nsteps)))


def wp_observe(h) -> np.ndarray:
    lib = load_library()
    o = WpObs()
    _check(lib, h, lib.wp_observe(h, ctypes.byref(o)))
    return _obs_array(ctypes.addressof(o), 1)[0]


def wp_run(h, nt: int, nprint: int) -> np.ndarray:
    lib = load_library()
    if nprint <= 0:
        raise ValueError("nprint must be > 0")
    cap = 1 + max(0, int(nt)) // int(nprint)
    buf = (WpObs * cap)()
    nobs = ctypes.c_int64(0)
    _check(lib, h, lib.wp_run(h, int(nt), int(nprint), ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(nobs)))
    return _obs_array(ctypes.addressof(buf), nobs.value)


def wp_fft(h, sign: int):
    lib = load_library()
    _check(lib, h, lib.wp_fft(h, int(sign)))


def wp_state_ptr(h) -> int:
    return load_library().wp_state_ptr(h) or 0


def wp_get_step_index(h) -> int:
    return load_library().wp_get_step_index(h)


def wp_set_step_index(h, s: int):
    lib = load_library()
    _check(lib, h, lib.wp_set_step_index(h, int(s)))


def wp_profile_enable(h, enable: bool):
    lib = load_library()
    _check(lib, h, lib.wp_profile_enable(h, 1 if enable else 0))


def wp_profile_read(h, kernel: int):
    lib = load_library()
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(lib, h, lib.wp_profile_read(h, int(kernel), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def wp_kernel_names():
    lib = load_library()
    return [lib.wp_kernel_name(i).decode() for i in range(lib.wp_kernel_count())]


def wp_launch_count(h) -> int:
    return load_library().wp_launch_count(h)


def _sched_dict(s: WpSchedule) -> dict:
    return {"tile_log": s.tile_log, "ept": s.ept, "max_radix_log": s.max_radix_log, "fixed": s.fixed}


def wp_get_schedule(h) -> dict:
    lib = load_library()
    s = WpSchedule()
    _check(lib, h, lib.wp_get_schedule(h, ctypes.byref(s)))
    return _sched_dict(s)


def wp_set_schedule(h, sched: dict):
    lib = load_library()
    s = WpSchedule(int(sched["tile_log"]), int(sched["ept"]), int(sched["max_radix_log"]), int(sched["fixed"]))
    _check(lib, h, lib.wp_set_schedule(h, ctypes.byref(s)))


def wp_autotune(h, steps: int = 3):
    """Times the candidate schedules, applies and caches the fastest; returns
    (schedule dict, ms per step, number of schedules timed)."""
    lib = load_library()
    s = WpSchedule()
    ms = ctypes.c_double(0.0)
    nc = ctypes.c_int32(0)
    _check(lib, h, lib.wp_autotune(h, int(steps), ctypes.byref(s), ctypes.byref(ms), ctypes.byref(nc)))
    return _sched_dict(s), ms.value, nc.value


def wp_autotune_cache_size() -> int:
    return load_library().wp_autotune_cache_size()


def wp_autotune_cache_clear():
    load_library().wp_autotune_cache_clear()


def wp_destroy(h):
    lib = load_library()
    lib.wp_destroy(h)


def _obs_array(addr, count):
    raw = (ctypes.c_char * (count * ctypes.sizeof(WpObs))).from_address(addr)
    return np.frombuffer(bytes(raw), dtype=OBS_DTYPE, count=count).copy()


def obs_matrix(obs: np.ndarray) -> np.ndarray:
    """Observation records as an [n, 16] float array in the oracle's column order."""
    cols = [obs[n].astype(np.float64) for n in OBS_DTYPE.names]
    return np.stack(cols, axis=-1)


# ---------------------------------------------------------------- convenience wrapper
def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Propagator:
    """One propagation on the GPU. problem/terms use the workloads.py schema."""

    def __init__(self, problem: dict, terms=(), precision="c128", autocorr=False, stream=None, mem_pool=None):
        self.problem = dict(problem)
        self.precision = precision
        self.shape = tuple(int(x) for x in problem["n"][: int(problem["ndim"])])
        self._pb = make_problem(problem, precision, autocorr)
        self.h = wp_create(self._pb, stream, mem_pool)
        if terms:
            self.set_potential(terms)

    def close(self):
        if getattr(self, "h", None):
            wp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_potential(self, terms):
        wp_set_potential(self.h, make_potential(list(terms)))

    def set_potential_grid(self, V):
        """Static potential on the grid: numpy float64 (host) or torch float64 CUDA tensor
        of the state's shape; None removes it."""
        if V is None:
            wp_set_potential_grid(self.h, None, False)
        elif hasattr(V, "is_cuda") and V.is_cuda:
            import torch
            t = V.contiguous().to(torch.float64)
            if tuple(t.shape) != self.shape:
                raise ValueError(f"grid shape {tuple(t.shape)} != {self.shape}")
            wp_set_potential_grid(self.h, t.data_ptr(), True)
        else:
            a = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
            if a.shape != self.shape:
                raise ValueError(f"grid shape {a.shape} != {self.shape}")
            wp_set_potential_grid(self.h, a.ctypes.data, False)

    def set_graphs(self, enable: bool):
        """CUDA-graph replay of repeated step(n) calls (needs a stream)."""
        wp_set_graphs(self.h, enable)

    def expect_grid(self, A) -> float:
        """<psi|A|psi> for a position-space operator on the grid (numpy or CUDA tensor)."""
        if hasattr(A, "is_cuda") and A.is_cuda:
            import torch
            t = A.contiguous().to(torch.float64)
            return wp_expect_grid(self.h, t.data_ptr(), True)
        a = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        if a.shape != self.shape:
            raise ValueError(f"operator shape {a.shape} != {self.shape}")
        return wp_expect_grid(self.h, a.ctypes.data, False)

    def run_with_callback(self, nt: int, nprint: int, fn):
        """Algorithm 1 with fn(propagator, record) called on every record (the state is
        the record's); a truthy return stops the run. Returns the records delivered."""
        return wp_run_callback(self.h, nt, nprint, lambda hp, rec: fn(self, rec))

    def set_potential_source(self, src: str):
        """CUDA C source defining __device__ double wp_user_potential(double x, double y,
        double z), compiled at run time and evaluated once on the grid."""
        wp_set_potential_source(self.h, src)

    @property
    def schedule(self) -> dict:
        return wp_get_schedule(self.h)

    def set_schedule(self, **sched):
        cur = wp_get_schedule(self.h)
        cur.update(sched)
        wp_set_schedule(self.h, cur)

    def autotune(self, steps: int = 3):
        return wp_autotune(self.h, steps)

    def init_gaussian(self, x0, p0, sigma):
        wp_init_gaussian(self.h, x0, p0, sigma)

    def set_state(self, psi):
        """psi: numpy complex128 array (host) or torch complex128 CUDA tensor (device)."""
        if hasattr(psi, "is_cuda") and psi.is_cuda:
            import torch
            t = psi.contiguous().to(torch.complex128)
            wp_set_state(self.h, t.data_ptr(), True)
            torch.cuda.current_stream().synchronize()
        else:
            a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.shape)
            wp_set_state(self.h, a.ctypes.data, False)

    def get_state(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        wp_get_state(self.h, out.ctypes.data, False)
        return out

    def get_state_device(self, out):
        """Copy the state as complex128 into a CUDA tensor `out` (device to device)."""
        wp_get_state(self.h, out.data_ptr(), True)
        return out

    def step(self, nsteps: int):
        wp_step(self.h, nsteps)

    def run(self, nt: int, nprint: int) -> np.ndarray:
        return wp_run(self.h, nt, nprint)

    def observe(self):
        return wp_observe(self.h)

    def fft(self, sign: int):
        wp_fft(self.h, sign)

    @property
    def step_index(self) -> int:
        return wp_get_step_index(self.h)

    @step_index.setter
    def step_index(self, s: int):
        wp_set_step_index(self.h, s)

    @property
    def launches(self) -> int:
        return wp_launch_count(self.h)

    def profile(self, enable: bool):
        wp_profile_enable(self.h, enable)

    def profile_read(self):
        names = wp_kernel_names()
        return {nm: wp_profile_read(self.h, i) for i, nm in enumerate(names)}


class Batch:
    """Many independent propagations advanced together (wp_batch_*)."""

    def __init__(self, precision="c128", stream=None):
        lib = load_library()
        self.lib = lib
        self.precision = precision
        h = ctypes.c_void_p()
        st = lib.wp_batch_create(PRECISIONS[precision], ctypes.c_void_p(stream or 0), ctypes.byref(h))
        _check(lib, None, st)
        self.b = h
        self.shapes = []
        self.problems = []

    def add(self, problem: dict, terms=(), autocorr=False) -> int:
        pb = make_problem(problem, self.precision, autocorr)
        pot = make_potential(list(terms))
        idx = ctypes.c_int64(-1)
        st = self.lib.wp_batch_add(self.b, ctypes.byref(pb), ctypes.byref(pot), ctypes.byref(idx))
        if st != WP_OK:
            raise WavepacketError(st, self.lib.wp_batch_last_error(self.b).decode(errors="replace"))
        self.shapes.append(tuple(int(x) for x in problem["n"][: int(problem["ndim"])]))
        self.problems.append(pb)
        return idx.value

    def handle(self, k: int):
        return ctypes.c_void_p(self.lib.wp_batch_handle(self.b, int(k)))

    def init_gaussian(self, k, x0, p0, sigma):
        wp_init_gaussian(self.handle(k), x0, p0, sigma)

    def set_state(self, k, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.shapes[k])
        wp_set_state(self.handle(k), a.ctypes.data, False)

    def get_state(self, k) -> np.ndarray:
        out = np.empty(self.shapes[k], dtype=np.complex128)
        wp_get_state(self.handle(k), out.ctypes.data, False)
        return out

    def step(self, nsteps: int, use_graph: bool = True):
        st = self.lib.wp_batch_step(self.b, int(nsteps), 1 if use_graph else 0)
        if st != WP_OK:
            raise WavepacketError(st, self.lib.wp_batch_last_error(self.b).decode(errors="replace"))

    @property
    def launches(self) -> int:
        return self.lib.wp_batch_launch_count(self.b)

    def __len__(self):
        return self.lib.wp_batch_size(self.b)

    def close(self):
        if getattr(self, "b", None):
            self.lib.wp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching request loop (wp_server_*)."""

    def __init__(self, budget_bytes=80e9, nslots=32, chunk_steps=50):
        lib = load_library()
        self.lib = lib
        h = ctypes.c_void_p()
        st = lib.wp_server_create(int(budget_bytes), int(nslots), int(chunk_steps), ctypes.byref(h))
        if st != WP_OK:
            raise WavepacketError(st, "wp_server_create failed")
        self.s = h
        self.shapes = {}
        self._done = (ctypes.c_int64 * 4096)()

    def _err(self, st):
        raise WavepacketError(st, self.lib.wp_server_last_error(self.s).decode(errors="replace"))

    def submit(self, rid: int, problem: dict, terms, init: dict, nt: int, precision="c64"):
        pb = make_problem(problem, precision)
        pot = make_potential(list(terms))
        st = self.lib.wp_server_submit(self.s, int(rid), ctypes.byref(pb), ctypes.byref(pot),
                                       _vec3(init["x0"], 0.0), _vec3(init["p0"], 0.0), _vec3(init["sigma"], 1.0),
                                       int(nt))
        if st != WP_OK:
            self._err(st)
        self.shapes[int(rid)] = tuple(int(x) for x in problem["n"][: int(problem["ndim"])])

    def progress(self):
        n = ctypes.c_int64(0)
        st = self.lib.wp_server_progress(self.s, self._done, len(self._done), ctypes.byref(n))
        if st != WP_OK:
            self._err(st)
        return [self._done[k] for k in range(min(n.value, len(self._done)))]

    def fetch(self, rid: int, want_state=False):
        psi = np.empty(self.shapes[rid], dtype=np.complex128) if want_state else None
        o = WpObs()
        times = (ctypes.c_double * 3)()
        st = self.lib.wp_server_fetch(self.s, int(rid), psi.ctypes.data if psi is not None else None,
                                      ctypes.byref(o), times)
        if st != WP_OK:
            self._err(st)
        del self.shapes[rid]
        return psi, _obs_array(ctypes.addressof(o), 1)[0], tuple(times)

    @property
    def pending(self) -> int:
        return self.lib.wp_server_pending(self.s)

    @property
    def running(self) -> int:
        return self.lib.wp_server_running(self.s)

    @property
    def bytes_in_use(self) -> int:
        return self.lib.wp_server_bytes_in_use(self.s)

    def close(self):
        if getattr(self, "s", None):
            self.lib.wp_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def problem_points(problem: dict) -> int:
    return int(math.prod(int(x) for x in problem["n"][: int(problem["ndim"])]))
