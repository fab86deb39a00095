"""Continuous-batching server: every request's result is the same alone and in the mix,
admission respects the memory budget, and the latency bookkeeping is consistent."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from paper_1306_3247_gb300 import serving as S
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_stream(count=14, seed=7):
    out = []
    for arr, job in W.request_stream(count=count, seed=seed):
        pb = dict(job["problem"])
        cap = {1: 4096, 2: 128, 3: 32}[pb["ndim"]]
        pb["n"] = [min(x, cap) for x in pb["n"]]
        nt = min(job["nt"], 120)
        out.append((arr, dict(job, problem=pb, nt=nt, nprint=nt)))
    return out


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_served_results_equal_alone(precision):
    reqs = small_stream()
    chunk = 25
    summary, results = S.serve(reqs, budget_bytes=2e9, nslots=4, chunk_steps=chunk, precision=precision,
                               time_scale=0.01, want_states=True)
    assert summary["requests"] == len(reqs) and len(results) == len(reqs)
    assert summary["p50_ms"] <= summary["p99_ms"]
    for rid, (arr, job) in enumerate(reqs):
        with WPK.Propagator(job["problem"], job["terms"], precision) as P:
            P.init_gaussian(**job["init"])
            left = job["nt"]
            while left > 0:
                m = min(chunk, left)
                P.step(m)
                left -= m
            alone = P.get_state()
            obs_alone = P.observe()
        obs, psi, lat = results[rid]
        assert np.array_equal(psi, alone), rid
        assert obs["norm"] == obs_alone["norm"] and obs["step"] == job["nt"]
        assert lat > 0


def test_budget_limits_concurrency():
    reqs = small_stream(count=8, seed=3)
    one = max(W_bytes for W_bytes in [2 ** 22])
    # a budget that fits only small requests one at a time still completes the stream
    summary, results = S.serve(reqs, budget_bytes=64e6, nslots=8, chunk_steps=40, time_scale=0.0)
    assert len(results) == len(reqs)
    with WPK.Server(1e6, 2, 10) as srv:
        big = W.config_3d_barrier(n=64)
        with pytest.raises(WPK.WavepacketError) as e:
            srv.submit(0, big["problem"], big["terms"], big["init"], 10)
        assert e.value.status == WPK.WP_ENOMEM


def _cudart():
    for cand in ("/usr/local/cuda/lib64/libcudart.so", ctypes.util.find_library("cudart")):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    pytest.skip("no CUDA runtime library to create a memory pool with")


class _PoolProps(ctypes.Structure):
    # cudaMemPoolProps: allocType, handleTypes, location {type, id}, win32 attributes,
    # maxSize, usage, reserved bytes
    _fields_ = [("allocType", ctypes.c_int), ("handleTypes", ctypes.c_int), ("loc_type", ctypes.c_int),
                ("loc_id", ctypes.c_int), ("win32", ctypes.c_void_p), ("maxSize", ctypes.c_size_t),
                ("usage", ctypes.c_ushort), ("reserved", ctypes.c_ubyte * 54)]


@pytest.mark.parametrize("precision", ["c64", "c128"])
def test_pooled_handle_equals_plain_handle(precision):
    """A handle whose device memory comes from the caller's stream-ordered pool
    (wp_create_pooled, what the server uses for admissions) gives the same bits as one
    from wp_create, and gives its memory back to the pool."""
    rt = _cudart()
    dev = ctypes.c_int(0)
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    props = _PoolProps()
    props.allocType = 1  # cudaMemAllocationTypePinned
    props.loc_type = 1   # cudaMemLocationTypeDevice
    props.loc_id = dev.value
    pool = ctypes.c_void_p()
    assert rt.cudaMemPoolCreate(ctypes.byref(pool), ctypes.byref(props)) == 0
    try:
        cfg = W.config_3d_barrier(n=64)
        outs = []
        for mp in (None, pool.value):
            with WPK.Propagator(cfg["problem"], cfg["terms"], precision, autocorr=True, mem_pool=mp) as P:
                P.init_gaussian(**cfg["init"])
                obs = P.run(40, 20)
                outs.append((P.get_state(), obs))
        assert np.array_equal(outs[0][0], outs[1][0])
        assert np.array_equal(WPK.obs_matrix(outs[0][1]), WPK.obs_matrix(outs[1][1]))
        used = ctypes.c_uint64(0)
        # cudaMemPoolAttrUsedMemCurrent = 7: nothing of the destroyed handle is still allocated
        assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0
        assert used.value == 0
    finally:
        rt.cudaDeviceSynchronize()
        rt.cudaMemPoolDestroy(pool)
