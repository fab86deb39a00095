"""Parity of the CUDA path with the FP64 CPU oracle at the bar the method is held to:
complex128 accuracy (native FP64 and float-float), relative L2 <= 1e-11 after 1000 steps
(the 2-D laser trap extended from 500 to 1000 steps on its full 1024^2 grid, the 3-D
barrier at 64^3 for 1000 steps) and after the 256^3 barrier job's full 200 steps;
complex64, relative L2 <= 2e-4 and norm drift <= 1e-5 on the same runs. Every
observable record (Tab. 3 quantities, autocorrelation included) is compared too.

The split step is eq. (splitop) of Sec. 2.1, chained as in Algorithm 1. Each oracle run
is computed once per module and shared by the three arithmetic forms.
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
DRIFT64 = 1e-5


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def compare_obs(obs, ref, rtol):
    M = WPK.obs_matrix(obs)
    assert M.shape == ref.shape
    assert np.array_equal(M[:, 15], ref[:, 15])
    assert np.allclose(M[:, 0], ref[:, 0], rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(ref[:, 0]))))
    scale = np.maximum(np.max(np.abs(ref[:, 1:15]), axis=0), 1e-300)
    err = np.max(np.abs(M[:, 1:15] - ref[:, 1:15]), axis=0) / np.maximum(scale, 1.0)
    assert np.all(err < rtol), err


_ORACLE = {}


def oracle_run(key, cfg, nt, nprint):
    """Final state and records of the oracle for one workload (cached per module)."""
    if key not in _ORACLE:
        pb, terms = cfg["problem"], cfg["terms"]
        psi0 = O.gaussian(pb, **cfg["init"])
        _ORACLE[key] = O.run(pb, terms, psi0, nt, nprint)
    return _ORACLE[key]


def gpu_run(cfg, prec, nt, nprint):
    with WPK.Propagator(cfg["problem"], cfg["terms"], prec, autocorr=True) as P:
        P.init_gaussian(**cfg["init"])
        obs = P.run(nt, nprint)
        psi = P.get_state()
        assert P.step_index == nt
    return psi, obs


def check(prec, psi, obs, ref, ref_obs):
    err = rel_l2(psi, ref)
    drift = float(np.max(np.abs(obs["norm"] - obs["norm"][0])))
    print(f"{prec}: relative L2 against the oracle {err:.3e}, norm drift {drift:.3e}")
    if prec == "c64":
        assert err < TOL64
        assert drift < DRIFT64
        compare_obs(obs, ref_obs, TOL64)
    else:
        assert err < TOL128
        compare_obs(obs, ref_obs, 1e-10)


# --------------------------------------------------------------------------- 3-D barrier, 64^3 x 1000
@pytest.mark.parametrize("prec", ["c128", "c128f", "c64"])
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_3d_barrier_64_cube_1000_steps(order, prec):
    cfg = W.config_3d_barrier(n=64, order=order)
    ref, ref_obs = oracle_run(("barrier64", order), cfg, 1000, 100)
    psi, obs = gpu_run(cfg, prec, 1000, 100)
    check(prec, psi, obs, ref, ref_obs)


# --------------------------------------------------------------------------- 3-D barrier, 256^3 x 200 (the full job)
@pytest.mark.parametrize("prec", ["c128", "c128f", "c64"])
def test_3d_barrier_256_cube_full_job(prec):
    cfg = W.config_3d_barrier(n=256)
    ref, ref_obs = oracle_run("barrier256", cfg, cfg["nt"], cfg["nprint"])
    psi, obs = gpu_run(cfg, prec, cfg["nt"], cfg["nprint"])
    check(prec, psi, obs, ref, ref_obs)


# --------------------------------------------------------------------------- 2-D laser trap, 1024^2 x 1000
@pytest.mark.parametrize("prec", ["c128", "c128f", "c64"])
def test_2d_laser_trap_1024_1000_steps(prec):
    cfg = W.config_2d_laser_trap(n=1024)
    ref, ref_obs = oracle_run("laser1024", cfg, 1000, 100)
    psi, obs = gpu_run(cfg, prec, 1000, 100)
    check(prec, psi, obs, ref, ref_obs)


# --------------------------------------------------------------------------- Sec. 4.2 Paul trap, SI units
def paul_small():
    cfg = W.config_paul_trap(n=64)
    cfg = dict(cfg, problem=dict(cfg["problem"], xmin=[-3.5e-7] * 3, L=[7e-7] * 3))
    return cfg


def compare_obs_si(obs, ref, rtol, mass):
    """Records in SI units: each column against its own physical scale (lengths against
    the packet width, momenta against the momentum spread, energies against the largest
    energy), since absolute values are of order 1e-8 m, 1e-27 kg m/s and 1e-29 J."""
    M = WPK.obs_matrix(obs)
    assert M.shape == ref.shape
    assert np.array_equal(M[:, 15], ref[:, 15])
    assert np.max(np.abs(M[:, 0] - ref[:, 0])) <= 1e-12 * np.max(np.abs(ref[:, 0]))
    assert np.max(np.abs(M[:, 1] - ref[:, 1])) < rtol
    assert np.max(np.abs(M[:, 14] - ref[:, 14])) < rtol
    pscale = math.sqrt(2.0 * mass * np.max(ref[:, 12]))
    for d in range(3):
        xscale = math.sqrt(np.max(ref[:, 8 + d]))
        assert np.max(np.abs(M[:, 2 + d] - ref[:, 2 + d])) < rtol * xscale
        assert np.max(np.abs(M[:, 5 + d] - ref[:, 5 + d])) < rtol * pscale
        assert np.max(np.abs(M[:, 8 + d] - ref[:, 8 + d])) < rtol * xscale ** 2
    escale = np.max(np.abs(ref[:, 11:14]))
    assert np.max(np.abs(M[:, 11:14] - ref[:, 11:14])) < rtol * escale


@pytest.mark.parametrize("prec", ["c128", "c128f", "c64"])
def test_paul_trap_64_cube_si_units_against_oracle(prec):
    """The Ba+ trap of Sec. 4.2 in SI units (hbar = 1.05e-34 J s, m = 2.3e-25 kg,
    dt = 2 ns) on a 64^3 grid around the packet: 60 steps, records every 10. In SI units
    k^2 |psi_hat|^2 is about 1e45, beyond the FP32 range the complex64 and float-float
    line sums are formed in: the kernels scale their coordinate and wavenumber tables."""
    cfg = paul_small()
    ref, ref_obs = oracle_run("paul64", cfg, 60, 10)
    psi, obs = gpu_run(cfg, prec, 60, 10)
    err = rel_l2(psi, ref)
    print(f"{prec}: relative L2 against the oracle {err:.3e}")
    assert err < (TOL64 if prec == "c64" else TOL128)
    compare_obs_si(obs, ref_obs, TOL64 if prec == "c64" else 1e-10, cfg["problem"]["mass"])


def verlet_moments(x, p, m, stiff, nt, dt, npr):
    out = []
    for s in range(nt):
        p = p - stiff(s * dt) * x * dt / 2
        x = x + p * dt / m
        p = p - stiff((s + 1) * dt) * x * dt / 2
        if (s + 1) % npr == 0:
            out.append((x, p))
    return out


def test_paul_trap_512_cube_full_run_follows_verlet():
    """The paper's whole Sec. 4.2 run: 512^3, 18 500 steps of 2 ns (one secular period),
    records every 10 steps, in the float-float complex128-accuracy form. The trap is
    quadratic with a periodic coefficient, so every <x_d>, <p_d> of the discrete method
    follows the Verlet map of x'' = -k(t) x / m exactly, up to rounding."""
    cfg = W.config_paul_trap(n=512)
    pb, terms = cfg["problem"], cfg["terms"]
    tm = terms[0]
    nt, npr = cfg["nt"], cfg["nprint"]
    with WPK.Propagator(pb, terms, "c128f") as P:
        P.init_gaussian(**cfg["init"])
        obs = P.run(nt, npr)
    M = WPK.obs_matrix(obs)
    assert M.shape[0] == 1 + nt // npr
    coef = lambda t: tm["coef"]["A0"] + tm["coef"]["A"] * math.sin(tm["coef"]["omega"] * t + tm["coef"]["phi"])
    for d in range(3):
        ref = np.array(verlet_moments(M[0, 2 + d], M[0, 5 + d], pb["mass"], lambda t, d=d: coef(t) * tm["a"][d],
                                      nt, pb["dt"], npr))
        ax, ap = np.max(np.abs(ref[:, 0])), max(np.max(np.abs(ref[:, 1])), 1e-30)
        ex = np.max(np.abs(M[1:, 2 + d] - ref[:, 0])) / ax
        ep = np.max(np.abs(M[1:, 5 + d] - ref[:, 1])) / ap
        print(f"axis {d}: amplitude {ax:.3e} m, {ap:.3e} kg m/s; max error {ex:.2e}, {ep:.2e}")
        assert ex < 1e-8 and ep < 1e-8
    # one secular period: the packet is back near its start (Fig. 2)
    assert np.max(np.abs(M[:, 1] - 1.0)) < 1e-9
