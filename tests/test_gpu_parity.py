"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: complex128 form, relative L2 <= 1e-11 after 1000 steps; complex64 form,
relative L2 <= 2e-4 and norm drift <= 1e-5 (the bounds the target states).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL128 = 1e-11
TOL64 = 2e-4


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    WPK.load_library()


def compare_obs(obs, ref, rtol):
    M = WPK.obs_matrix(obs)
    assert M.shape == ref.shape
    assert np.array_equal(M[:, 15], ref[:, 15])
    assert np.allclose(M[:, 0], ref[:, 0], rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(ref[:, 0]))))
    scale = np.maximum(np.max(np.abs(ref[:, 1:15]), axis=0), 1e-300)
    err = np.max(np.abs(M[:, 1:15] - ref[:, 1:15]), axis=0) / np.maximum(scale, 1.0)
    assert np.all(err < rtol), err


# --------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("shape", [(2,), (8,), (64,), (1024,), (4096,), (8192,), (2, 4), (64, 32), (8, 1024),
                                   (4, 8, 16), (16, 16, 16), (2, 64, 8), (32, 2, 256)])
@pytest.mark.parametrize("prec", ["c128", "c64", "c128f"])
def test_fft_matches_oracle(shape, prec):
    nd = len(shape)
    pb = {"ndim": nd, "n": list(shape), "xmin": [0.0] * nd, "L": [1.0] * nd, "dt": 0.1}
    x = W.random_state(shape, seed=sum(shape))
    tol = {"c128": 1e-13, "c64": 3e-6, "c128f": 1e-12}[prec]
    with WPK.Propagator(pb, precision=prec) as P:
        P.set_state(x)
        P.fft(-1)
        X = P.get_state()
        assert rel_l2(X, O.fft(x, -1)) < tol
        P.fft(+1)
        assert rel_l2(P.get_state(), O.fft(O.fft(x, -1), +1)) < tol
        assert rel_l2(P.get_state() / x.size, x) < tol


# Shapes that run the two-stage kernels for 256-point lines: the contiguous axis with 8
# (float-float) or 16 (complex64) lines or more, and strided axes with as many adjacent
# columns; smaller ones keep the Stockham kernels. Native complex128 runs every shape on
# the Stockham kernels.
@pytest.mark.parametrize("shape", [(16, 256), (256, 16), (256, 256), (4, 256, 32), (256, 2, 16), (2, 256, 64),
                                   (8, 256), (256, 8), (256, 4, 2)])
@pytest.mark.parametrize("prec", ["c64", "c128f", "c128"])
def test_fft_256_lines_match_oracle(shape, prec):
    nd = len(shape)
    pb = {"ndim": nd, "n": list(shape), "xmin": [0.0] * nd, "L": [1.0] * nd, "dt": 0.1}
    x = W.random_state(shape, seed=7 * sum(shape))
    tol = {"c128": 1e-13, "c64": 3e-6, "c128f": 1e-12}[prec]
    with WPK.Propagator(pb, precision=prec) as P:
        P.set_state(x)
        P.fft(-1)
        assert rel_l2(P.get_state(), O.fft(x, -1)) < tol
        P.fft(+1)
        assert rel_l2(P.get_state() / x.size, x) < tol


# Shapes that run the two-stage complex64 kernels for 64- and 128-point lines (32 lines or
# columns per tile for 64, 16 for 128), and smaller ones that keep the Stockham kernels.
@pytest.mark.parametrize("shape", [(32, 64), (64, 32), (16, 128), (128, 16), (64, 64), (128, 128), (64, 128),
                                   (2, 64, 32), (32, 2, 64), (4, 128, 16), (16, 64), (64, 16)])
def test_fft_64_128_lines_match_oracle_c64(shape):
    nd = len(shape)
    pb = {"ndim": nd, "n": list(shape), "xmin": [0.0] * nd, "L": [1.0] * nd, "dt": 0.1}
    x = W.random_state(shape, seed=11 * sum(shape))
    with WPK.Propagator(pb, precision="c64") as P:
        P.set_state(x)
        P.fft(-1)
        assert rel_l2(P.get_state(), O.fft(x, -1)) < 3e-6
        P.fft(+1)
        assert rel_l2(P.get_state() / x.size, x) < 3e-6


@pytest.mark.parametrize("shape", [(64, 64), (128, 64), (64, 128)])
def test_2d_64_128_c64_1000_steps(shape):
    # 64- and 128-point axes on the two-stage complex64 kernels: driven trap plus barrier
    pb = {"ndim": 2, "n": list(shape), "xmin": [-12.0, -10.0], "L": [24.0, 20.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.005, "t0": 0.0}
    terms = [{"shape": "quad", "a": [0.5, 0.8], "coef": {"A0": 1.0}},
             {"shape": "gauss", "a": [1.0, 1.2], "c0": [1.0, 0.0], "coef": {"A0": 1.0, "A": 0.3, "omega": 2.0}},
             {"shape": "linear", "a": [1.0, 0.0], "coef": {"A": 0.1, "omega": 0.7}}]
    psi0 = O.gaussian(pb, [-2.0, 0.5], [1.0, 0.0], [1.2, 1.0])
    ref, ref_obs = O.run(pb, terms, psi0, 1000, 100)
    with WPK.Propagator(pb, terms, "c64", autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(1000, 100)
        psi = P.get_state()
    err = rel_l2(psi, ref)
    drift = float(np.max(np.abs(obs["norm"] - obs["norm"][0])))
    print("c64", shape, "rel L2", err, "norm drift", drift)
    assert err < TOL64
    assert drift < 1e-5
    compare_obs(obs, ref_obs, TOL64)


def test_2d_256_square_c128f_1000_steps():
    # 256^2 on the two-stage float-float kernels, at the complex128 bar
    pb = {"ndim": 2, "n": [256, 256], "xmin": [-16.0, -16.0], "L": [32.0, 32.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.005, "t0": 0.0}
    terms = [{"shape": "quad", "a": [0.25, 0.5], "coef": {"A0": 1.0}},
             {"shape": "gauss", "a": [1.0, 1.5], "c0": [1.0, 0.0], "coef": {"A0": 1.0, "A": 0.3, "omega": 2.0}},
             {"shape": "linear", "a": [1.0, 0.0], "coef": {"A": 0.1, "omega": 0.7}}]
    psi0 = O.gaussian(pb, [-2.0, 0.5], [1.5, 0.0], [1.2, 1.0])
    ref, ref_obs = O.run(pb, terms, psi0, 1000, 100)
    with WPK.Propagator(pb, terms, "c128f", autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(1000, 100)
        psi = P.get_state()
    err = rel_l2(psi, ref)
    print("c128f 256^2 rel L2", err)
    assert err < TOL128
    compare_obs(obs, ref_obs, 1e-10)


def test_2d_256_square_c64_1000_steps():
    # 256^2: both axes on the two-stage complex64 kernels (contiguous: IFFT, phase, FFT;
    # strided: FFT, kinetic factor, IFFT), a Gaussian barrier and a driven trap
    pb = {"ndim": 2, "n": [256, 256], "xmin": [-16.0, -16.0], "L": [32.0, 32.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.005, "t0": 0.0}
    terms = [{"shape": "quad", "a": [0.25, 0.5], "coef": {"A0": 1.0}},
             {"shape": "gauss", "a": [1.0, 1.5], "c0": [1.0, 0.0], "coef": {"A0": 1.0, "A": 0.3, "omega": 2.0}},
             {"shape": "linear", "a": [1.0, 0.0], "coef": {"A": 0.1, "omega": 0.7}}]
    psi0 = O.gaussian(pb, [-2.0, 0.5], [1.5, 0.0], [1.2, 1.0])
    ref, ref_obs = O.run(pb, terms, psi0, 1000, 100)
    with WPK.Propagator(pb, terms, "c64", autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(1000, 100)
        psi = P.get_state()
    err = rel_l2(psi, ref)
    drift = float(np.max(np.abs(obs["norm"] - obs["norm"][0])))
    print("c64 256^2 rel L2", err, "norm drift", drift)
    assert err < TOL64
    assert drift < 1e-5
    compare_obs(obs, ref_obs, TOL64)


# --------------------------------------------------------------------------- 1-D
@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_1d_driven_trap_c128_1000_steps(order, prec):
    cfg = W.config_1d_driven_trap(order=order)
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, cfg["nt"], cfg["nprint"])
    with WPK.Propagator(pb, terms, prec, autocorr=True) as P:
        P.init_gaussian(**cfg["init"])
        assert rel_l2(P.get_state(), psi0) < (1e-15 if prec == "c128" else 1e-14)
        obs = P.run(cfg["nt"], cfg["nprint"])
        psi = P.get_state()
        assert P.step_index == cfg["nt"]
    assert rel_l2(psi, ref) < TOL128
    compare_obs(obs, ref_obs, 1e-10)


def test_1d_longest_line_c64():
    # 1-D complex64 lines go up to 16384 points (one resident block of 1024 threads)
    pb = {"ndim": 1, "n": [16384], "xmin": [-40.0], "L": [80.0], "dt": 0.005, "t0": 0.0}
    terms = [{"shape": "quad", "a": [0.25], "coef": {"A0": 1.0}},
             {"shape": "linear", "a": [1.0], "coef": {"A": 0.1, "omega": 0.45}}]
    psi0 = O.gaussian(pb, [1.0], [0.5], [1.5])
    ref = O.propagate(pb, terms, psi0, 200)
    with WPK.Propagator(pb, terms, "c64") as P:
        P.set_state(psi0)
        P.step(120)
        P.step(80)
        assert rel_l2(P.get_state(), ref) < TOL64


def test_1d_driven_trap_c64_1000_steps():
    cfg = W.config_1d_driven_trap()
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, cfg["nt"], cfg["nprint"])
    with WPK.Propagator(pb, terms, "c64") as P:
        P.set_state(psi0)
        obs = P.run(cfg["nt"], cfg["nprint"])
        psi = P.get_state()
    err = rel_l2(psi, ref)
    print("c64 1d rel L2", err, "norm drift", abs(obs["norm"][-1] - obs["norm"][0]))
    assert err < TOL64
    assert np.max(np.abs(obs["norm"] - obs["norm"][0])) < 1e-5


@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("n", [2, 4, 16, 256, 2048, 8192])
def test_1d_sizes_and_chunking(n, prec):
    pb = {"ndim": 1, "n": [n], "xmin": [-10.0], "L": [20.0], "mass": 1.3, "hbar": 0.9, "dt": 0.003, "t0": 0.25}
    terms = [{"shape": "gauss", "a": [1.2], "c0": [0.5], "v": [0.3], "coef": {"A0": 0.8, "A": 0.2, "omega": 1.1}},
             {"shape": "quad", "a": [0.5], "coef": {"A0": 1.0}}]
    psi0 = W.random_state((n,), seed=n)
    ref = O.propagate(pb, terms, psi0, 23)
    with WPK.Propagator(pb, terms, prec) as P:
        P.set_state(psi0)
        P.step(7)
        P.step(1)
        P.step(15)
        assert P.step_index == 23
        assert rel_l2(P.get_state(), ref) < TOL128


# --------------------------------------------------------------------------- 2-D
def small_laser_trap(n=128, order="vkv"):
    cfg = W.config_2d_laser_trap(n=n, order=order)
    pb = dict(cfg["problem"], xmin=[-10.0, -10.0], L=[20.0, 20.0])
    return cfg, pb


@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_2d_laser_trap_c128(order, prec):
    cfg, pb = small_laser_trap(order=order)
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, 200, 50)
    with WPK.Propagator(pb, terms, prec, autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(200, 50)
        psi = P.get_state()
    assert rel_l2(psi, ref) < TOL128
    compare_obs(obs, ref_obs, 1e-10)


def test_2d_laser_trap_c64():
    cfg, pb = small_laser_trap()
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, 1000, 100)
    with WPK.Propagator(pb, terms, "c64", autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(1000, 100)
        psi = P.get_state()
    assert rel_l2(psi, ref) < TOL64
    assert np.max(np.abs(obs["norm"] - obs["norm"][0])) < 1e-5
    compare_obs(obs, ref_obs, TOL64)


@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("shape", [(2, 2), (4, 1024), (2048, 4), (64, 128)])
def test_2d_shapes_random_state(shape, prec):
    pb = {"ndim": 2, "n": list(shape), "xmin": [-4.0, -6.0], "L": [8.0, 12.0], "mass": 0.7, "hbar": 1.0,
          "dt": 0.01, "t0": 0.0}
    terms = [{"shape": "quad", "a": [1.0, 0.5], "coef": {"A0": 1.0, "A": 0.3, "omega": 2.0}},
             {"shape": "gauss", "a": [1.0, 2.0], "c0": [0.3, -0.2], "coef": {"A0": 1.5}},
             {"shape": "linear", "a": [0.2, -0.1], "coef": {"A": 1.0, "omega": 0.7, "env": "gauss", "t0": 0.05,
                                                           "tau": 0.1}}]
    psi0 = W.random_state(shape, seed=3)
    ref = O.propagate(pb, terms, psi0, 12)
    with WPK.Propagator(pb, terms, prec) as P:
        P.set_state(psi0)
        P.step(5)
        P.step(7)
        assert rel_l2(P.get_state(), ref) < TOL128


# --------------------------------------------------------------------------- 3-D
def small_barrier(n=64, order="vkv"):
    cfg = W.config_3d_barrier(n=n, order=order)
    return cfg, cfg["problem"]


@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_3d_barrier_c128(order, prec):
    cfg, pb = small_barrier(order=order)
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, 60, 20)
    with WPK.Propagator(pb, terms, prec, autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(60, 20)
        psi = P.get_state()
    assert rel_l2(psi, ref) < TOL128
    compare_obs(obs, ref_obs, 1e-10)


def test_3d_barrier_c64():
    cfg, pb = small_barrier()
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, 200, 50)
    with WPK.Propagator(pb, terms, "c64", autocorr=True) as P:
        P.set_state(psi0)
        obs = P.run(200, 50)
        psi = P.get_state()
    assert rel_l2(psi, ref) < TOL64
    assert np.max(np.abs(obs["norm"] - obs["norm"][0])) < 1e-5
    compare_obs(obs, ref_obs, TOL64)


@pytest.mark.parametrize("prec", ["c128", "c128f"])
@pytest.mark.parametrize("shape", [(2, 2, 2), (4, 8, 16), (16, 4, 2), (8, 2, 512)])
def test_3d_shapes_random_state(shape, prec):
    pb = {"ndim": 3, "n": list(shape), "xmin": [-3.0, -4.0, -5.0], "L": [6.0, 8.0, 10.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.02, "t0": 0.1}
    terms = [{"shape": "quad", "a": [1.0, 2.0, 0.5], "coef": {"A0": 1.0}},
             {"shape": "gauss", "a": [1.0, 0.0, 2.0], "c0": [0.1, 0.0, -0.3], "v": [0.2, 0.0, 0.0],
              "coef": {"A0": 2.0, "A": 0.5, "omega": 3.0}},
             {"shape": "morse", "a": [0.3, 1.1, 2.0], "c0": [0.0, 0.0, 0.5], "coef": {"A0": 1.0}}]
    psi0 = W.random_state(shape, seed=5)
    ref = O.propagate(pb, terms, psi0, 9)
    with WPK.Propagator(pb, terms, prec) as P:
        P.set_state(psi0)
        P.step(9)
        assert rel_l2(P.get_state(), ref) < TOL128


# --------------------------------------------------------------------------- API rules
def test_status_errors():
    pb = {"ndim": 1, "n": [100], "xmin": [0.0], "L": [1.0], "dt": 0.1}
    with pytest.raises(WPK.WavepacketError) as e:
        WPK.Propagator(pb)
    assert e.value.status == WPK.WP_EUNSUPPORTED
    pb = {"ndim": 1, "n": [64], "xmin": [0.0], "L": [1.0], "dt": 0.1}
    with WPK.Propagator(pb) as P:
        with pytest.raises(WPK.WavepacketError) as e:
            P.run(5, 6)
        assert e.value.status == WPK.WP_EINVAL


def test_nonfinite_state_reported():
    pb = {"ndim": 2, "n": [16, 16], "xmin": [0.0, 0.0], "L": [1.0, 1.0], "dt": 0.1}
    psi = np.ones((16, 16), dtype=np.complex128)
    psi[3, 4] = np.nan
    with WPK.Propagator(pb) as P:
        P.set_state(psi)
        with pytest.raises(WPK.WavepacketError) as e:
            P.run(2, 1)
        assert e.value.status == WPK.WP_ENONFINITE


def test_observe_and_resume_match_uninterrupted_run():
    cfg = W.config_1d_driven_trap()
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    with WPK.Propagator(pb, terms) as P:
        P.set_state(psi0)
        P.step(100)
        chk = P.get_state()
        s = P.step_index
        P.step(50)
        full = P.get_state()
    with WPK.Propagator(pb, terms) as Q:
        Q.set_state(chk)
        Q.step_index = s
        Q.step(50)
        assert np.array_equal(Q.get_state(), full)
