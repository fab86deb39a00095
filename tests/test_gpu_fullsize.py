"""Parity at the workloads' full sizes, in the launch configuration bench.py times:
whole-array comparison with the oracle for a few steps, and properties that hold at any
size (exact Verlet moments for quadratic potentials, norm conservation) for full runs."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c128f", 1e-12), ("c64", 2e-5)])
def test_3d_barrier_256_cube_against_oracle(prec, tol):
    cfg = W.config_3d_barrier(n=256)
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref, ref_obs = O.run(pb, terms, psi0, 4, 2)
    with WPK.Propagator(pb, terms, prec) as P:
        P.init_gaussian(**cfg["init"])
        obs = P.run(4, 2)
        psi = P.get_state()
    assert rel_l2(psi, ref) < tol
    M = WPK.obs_matrix(obs)
    assert np.max(np.abs(M[:, 1] - ref_obs[:, 1])) < (1e-12 if prec != "c64" else 1e-6)
    assert np.max(np.abs(M[:, 11] - ref_obs[:, 11])) < (1e-10 if prec != "c64" else 1e-5) * abs(ref_obs[0, 11])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_2d_laser_trap_1024_against_oracle(prec):
    cfg = W.config_2d_laser_trap(n=1024)
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    ref = O.propagate(pb, terms, psi0, 10)
    with WPK.Propagator(pb, terms, prec) as P:
        P.init_gaussian(**cfg["init"])
        P.step(10)
        assert rel_l2(P.get_state(), ref) < (1e-12 if prec == "c128" else 2e-5)


def verlet_moments(x, p, m, stiff, force, nt, dt, npr):
    out = []
    for s in range(nt):
        p = p - (stiff(s * dt) * x + force(s * dt)) * dt / 2
        x = x + p * dt / m
        p = p - (stiff((s + 1) * dt) * x + force((s + 1) * dt)) * dt / 2
        if (s + 1) % npr == 0:
            out.append((x, p))
    return out


@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c128f", 1e-10), ("c64", 2e-5)])
def test_2d_laser_trap_full_run_follows_verlet(prec, tol):
    # full 1024^2 grid, all 500 steps: the moments follow the exact discrete Verlet map
    cfg = W.config_2d_laser_trap(n=1024)
    pb, terms = cfg["problem"], cfg["terms"]
    with WPK.Propagator(pb, terms, prec) as P:
        P.init_gaussian(**cfg["init"])
        obs = P.run(cfg["nt"], cfg["nprint"])
    M = WPK.obs_matrix(obs)
    fx = lambda t: 0.05 * math.exp(-((t - 10.0) / 4.0) ** 2) * math.sin(0.5 * t + W.HALF_PI)
    for d, (stiff, force) in enumerate([(lambda t: 1.0, fx), (lambda t: 4.0, lambda t: 0.0)]):
        ref = verlet_moments(M[0, 2 + d], M[0, 5 + d], 1.0, stiff, force, cfg["nt"], pb["dt"], cfg["nprint"])
        for k, (x, p) in enumerate(ref):
            assert abs(M[k + 1, 2 + d] - x) < tol and abs(M[k + 1, 5 + d] - p) < tol, (d, k)
    assert np.max(np.abs(M[:, 1] - M[0, 1])) < (1e-12 if prec != "c64" else 1e-5)


@pytest.mark.parametrize("prec", ["c128f", "c128"])
def test_paul_trap_512_cube_si_units_follows_verlet(prec):
    """The Ba+ Paul-trap run of Sec. 4.2 on its printed 512^3 grid in SI units: the trap is
    quadratic with a periodic coefficient, so each <x_d>, <p_d> follows the Verlet map."""
    cfg = W.config_paul_trap(n=512)
    pb, terms = cfg["problem"], cfg["terms"]
    tm = terms[0]
    nt, npr = 20, 10
    with WPK.Propagator(pb, terms, prec) as P:
        P.init_gaussian(**cfg["init"])
        obs = P.run(nt, npr)
    M = WPK.obs_matrix(obs)
    coef = lambda t: tm["coef"]["A0"] + tm["coef"]["A"] * math.sin(tm["coef"]["omega"] * t + tm["coef"]["phi"])
    for d in range(3):
        ref = verlet_moments(M[0, 2 + d], M[0, 5 + d], pb["mass"], lambda t, d=d: coef(t) * tm["a"][d],
                             lambda t: 0.0, nt, pb["dt"], npr)
        for k, (x, p) in enumerate(ref):
            assert abs(M[k + 1, 2 + d] - x) < 1e-9 * abs(x)
            assert abs(M[k + 1, 5 + d] - p) < 1e-9 * max(abs(p), 1e-27)
    assert np.max(np.abs(M[:, 1] - 1.0)) < 1e-10
