"""Pins for the FP64 CPU oracle: checks against things the oracle does not compute itself
(brute-force DFTs, closed forms, exact discrete maps, invariants, the paper's printed
parameters). A plausible slip in the oracle -- a dropped term, a wrong sign, a wrong
wavenumber ordering, a transposed axis, the wrong time for V -- fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(j, j) % n) / n)


def grid(pb, d):
    return pb["xmin"][d] + np.arange(pb["n"][d]) * (pb["L"][d] / pb["n"][d])


# --------------------------------------------------------------------------- FFT (eq. ft)
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_bruteforce_dft(n, sign):
    x = W.random_state((n,), seed=100 + n)
    ref = dft_matrix(n, sign) @ x
    assert rel_l2(O.fft(x, sign), ref) < 1e-14


def test_fft_3d_matches_bruteforce_per_axis():
    # distinct extents so that a transposed axis or a wrong stride fails
    x = W.random_state((4, 8, 16), seed=7)
    ref = np.einsum("ia,abc->ibc", dft_matrix(4, -1), x)
    ref = np.einsum("jb,ibc->ijc", dft_matrix(8, -1), ref)
    ref = np.einsum("kc,ijc->ijk", dft_matrix(16, -1), ref)
    assert rel_l2(O.fft(x, -1), ref) < 1e-14
    # library routine as a second, independent check
    assert rel_l2(O.fft(x, -1), np.fft.fftn(x)) < 1e-14


@pytest.mark.parametrize("shape", [(1024,), (64, 32), (16, 8, 32)])
def test_fft_roundtrip_and_parseval(shape):
    x = W.random_state(shape, seed=11)
    X = O.fft(x, -1)
    N = x.size
    assert abs(np.vdot(X, X).real / N - np.vdot(x, x).real) / np.vdot(x, x).real < 1e-14
    assert rel_l2(O.fft(X, +1) / N, x) < 1e-15 * 10


# --------------------------------------------------------------------------- closed forms
def free_gaussian_1d(x, t, x0, p0, sigma, m, hbar):
    """Free-particle evolution of the Sec. 4.2 packet (position std s = sigma/2)."""
    s = sigma / 2.0
    k0 = p0 / hbar
    T = 2.0 * m * s * s / hbar
    a = 1.0 + 1j * t / T
    v = hbar * k0 / m
    return ((2 * np.pi * s * s) ** -0.25 / np.sqrt(a)
            * np.exp(-(x - x0 - v * t) ** 2 / (4 * s * s * a) + 1j * k0 * (x - x0)
                     - 1j * hbar * k0 * k0 * t / (2 * m)))


@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_free_gaussian_closed_form_1d(order):
    pb = {"ndim": 1, "n": [1024], "xmin": [-20.0], "L": [40.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.01, "t0": 0.0, "order": order}
    psi0 = O.gaussian(pb, [-5.0], [2.0], [1.0])
    x = grid(pb, 0)
    assert rel_l2(psi0, free_gaussian_1d(x, 0.0, -5.0, 2.0, 1.0, 1.0, 1.0)) < 1e-14
    psi = O.propagate(pb, [], psi0, 100)  # t = 1: the spread packet stays clear of the box edge
    ref = free_gaussian_1d(x, 1.0, -5.0, 2.0, 1.0, 1.0, 1.0)
    assert rel_l2(psi, ref) < 1e-12


def test_free_gaussian_closed_form_3d_anisotropic():
    # different n, L, mass, hbar, p0 per axis: catches swapped axes or wavenumber grids
    pb = {"ndim": 3, "n": [64, 64, 128], "xmin": [-12.0, -12.0, -16.0], "L": [24.0, 24.0, 32.0],
          "mass": 1.7, "hbar": 0.8, "dt": 0.02, "t0": 0.0, "order": "vkv"}
    x0, p0, sg = [-1.0, 0.5, 2.0], [1.2, -0.7, 0.0], [1.6, 1.9, 1.3]
    psi0 = O.gaussian(pb, x0, p0, sg)
    psi = O.propagate(pb, [], psi0, 25)
    t = 0.5
    f = [free_gaussian_1d(grid(pb, d), t, x0[d], p0[d], sg[d], 1.7, 0.8) for d in range(3)]
    ref = f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
    assert rel_l2(psi, ref) < 1e-11


def free_gaussian_autocorr(t, p0, sigma, m, hbar):
    """|<psi(0)|psi(t)>|^2 of a free Sec. 4.2 packet along one axis. Its wavenumber is
    normally distributed, mean k0 = p0/hbar and variance 1/sigma^2 (position std sigma/2),
    and the free evolution multiplies each wavenumber component by exp(-i a k^2) with
    a = hbar t / 2m, so the overlap is the characteristic function of a noncentral
    chi-square: (1 + 2 i a s2)^(-1/2) exp(-i a k0^2 / (1 + 2 i a s2)), s2 = 1/sigma^2.
    Its squared modulus is (1 + 4 a^2 s2^2)^(-1/2) exp(-4 a^2 s2 k0^2 / (1 + 4 a^2 s2^2))."""
    s2 = 1.0 / (sigma * sigma)
    k0 = p0 / hbar
    a = hbar * t / (2.0 * m)
    q = 1.0 + 4.0 * a * a * s2 * s2
    return q ** -0.5 * math.exp(-4.0 * a * a * s2 * k0 * k0 / q)


@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_free_gaussian_autocorrelation_closed_form_1d(order):
    # Tab. 3 autocorrelation |<psi(0)|psi(t)>|^2 at t > 0: a moving, spreading packet whose
    # overlap with psi(0) falls from 1 to 0.096 by t = 1 (ground states would stay at 1)
    pb = {"ndim": 1, "n": [1024], "xmin": [-20.0], "L": [40.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.01, "t0": 0.0, "order": order}
    psi0 = O.gaussian(pb, [-5.0], [2.0], [1.0])
    _, obs = O.run(pb, [], psi0, 100, 20)
    assert len(obs) == 6 and obs[-1, 14] < 0.1
    for rec in obs:
        assert abs(rec[14] - free_gaussian_autocorr(rec[0], 2.0, 1.0, 1.0, 1.0)) < 1e-12, rec[0]


def test_free_gaussian_autocorrelation_closed_form_3d_anisotropic():
    # the overlap of a product state is the product of the per-axis overlaps; different
    # n, L, mass, hbar, p0 and sigma per axis, and a nonzero t0
    pb = {"ndim": 3, "n": [64, 64, 128], "xmin": [-12.0, -12.0, -16.0], "L": [24.0, 24.0, 32.0],
          "mass": 1.7, "hbar": 0.8, "dt": 0.04, "t0": 0.3, "order": "kvk"}
    x0, p0, sg = [-1.0, 0.5, 2.0], [1.2, -0.7, 0.0], [1.6, 1.9, 1.3]
    psi0 = O.gaussian(pb, x0, p0, sg)
    _, obs = O.run(pb, [], psi0, 30, 10)
    for rec in obs:
        t = rec[0] - pb["t0"]
        ref = math.prod(free_gaussian_autocorr(t, p0[d], sg[d], 1.7, 0.8) for d in range(3))
        assert abs(rec[14] - ref) < 1e-12, t
    assert obs[-1, 14] < 0.8


@pytest.mark.parametrize("j", [3, 64 - 5, 32])
def test_plane_wave_kinetic_phase_and_momentum(j):
    # psi = exp(i k_j x) with k_j from the FFT ordering (j >= n/2 is negative; n/2 is Nyquist)
    n, L, m, hbar, dt = 64, 10.0, 1.3, 0.9, 0.07
    pb = {"ndim": 1, "n": [n], "xmin": [-3.0], "L": [L], "mass": m, "hbar": hbar, "dt": dt,
          "t0": 0.0, "order": "vkv"}
    js = j if j < n // 2 else j - n
    k = 2 * np.pi * js / L
    x = grid(pb, 0)
    psi0 = np.exp(1j * k * x)
    psi1 = O.step(pb, [], psi0)
    assert rel_l2(psi1, np.exp(-1j * hbar * k * k * dt / (2 * m)) * psi0) < 1e-13
    rec = O.observe(pb, [], psi0)
    assert abs(rec[5] - hbar * k * L) < 1e-11 * max(1.0, abs(hbar * k * L))
    assert abs(rec[12] - hbar ** 2 * k * k / (2 * m) * L) < 1e-11 * max(1.0, hbar ** 2 * k * k * L)


def test_harmonic_ground_state_energy_and_width():
    m, hbar, w = 0.9, 1.1, 1.3
    pb = {"ndim": 1, "n": [256], "xmin": [-16.0], "L": [32.0], "mass": m, "hbar": hbar,
          "dt": 0.01, "t0": 0.0, "order": "vkv"}
    terms = [{"shape": "quad", "a": [m * w * w], "coef": {"A0": 1.0}}]
    sigma = math.sqrt(2 * hbar / (m * w))
    psi0 = O.gaussian(pb, [0.0], [0.0], [sigma])
    rec = O.observe(pb, terms, psi0, psi0)
    assert abs(rec[1] - 1.0) < 1e-13
    assert abs(rec[11] - hbar * w / 2) < 1e-12
    assert abs(rec[12] - hbar * w / 4) < 1e-12  # virial: E_K = E_V
    assert abs(rec[8] - sigma ** 2 / 4) < 1e-12
    assert abs(rec[14] - 1.0) < 1e-12
    # stationarity: density and energy move only at O(dt^2)
    psi, obs = O.run(pb, terms, psi0, 400, 100)
    assert np.max(np.abs(np.abs(psi) ** 2 - np.abs(psi0) ** 2)) < 1e-4
    assert np.max(np.abs(obs[:, 11] - hbar * w / 2)) < 1e-4
    assert np.max(np.abs(obs[:, 1] - 1.0)) < 1e-13


def test_harmonic_ground_state_3d_anisotropic_energy():
    w = [1.0, 2.0, 0.5]
    pb = {"ndim": 3, "n": [32, 32, 32], "xmin": [-8.0, -6.0, -12.0], "L": [16.0, 12.0, 24.0],
          "mass": 1.0, "hbar": 1.0, "dt": 0.01, "t0": 0.0, "order": "vkv"}
    terms = [{"shape": "quad", "a": [ww * ww for ww in w], "coef": {"A0": 1.0}}]
    sg = [math.sqrt(2.0 / ww) for ww in w]
    rec = O.observe(pb, terms, O.gaussian(pb, [0.0] * 3, [0.0] * 3, sg))
    assert abs(rec[11] - sum(w) / 2) < 1e-11
    for d in range(3):
        assert abs(rec[8 + d] - sg[d] ** 2 / 4) < 1e-11


# --------------------------------------------------------------------------- exact discrete maps
def verlet_vkv(x, p, m, stiff, force, times, dt):
    """Velocity Verlet: the exact image of the VKV step on (<x>, <p>) for V = stiff x^2/2 + force(t) x."""
    p = p - (stiff * x + force(times[0])) * dt / 2
    x = x + p * dt / m
    p = p - (stiff * x + force(times[1])) * dt / 2
    return x, p


def verlet_kvk(x, p, m, stiff, force, tmid, dt):
    """Position Verlet: the exact image of the paper's KVK step (V at the midpoint)."""
    x = x + p * dt / (2 * m)
    p = p - (stiff * x + force(tmid)) * dt
    x = x + p * dt / (2 * m)
    return x, p


@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_driven_trap_1d_follows_verlet_map(order):
    cfg = W.config_1d_driven_trap(order=order)
    pb, terms = cfg["problem"], cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    psi, obs = O.run(pb, terms, psi0, cfg["nt"], cfg["nprint"])
    dt = pb["dt"]
    force = lambda t: 0.1 * math.sin(0.9 * t)
    x, p = obs[0, 2], obs[0, 5]
    assert abs(x - 2.0) < 1e-12 and abs(p) < 1e-12
    for s in range(cfg["nt"]):
        if order == "vkv":
            x, p = verlet_vkv(x, p, 1.0, 1.0, force, (s * dt, (s + 1) * dt), dt)
        else:
            x, p = verlet_kvk(x, p, 1.0, 1.0, force, s * dt + dt / 2, dt)
        if (s + 1) % cfg["nprint"] == 0:
            r = obs[(s + 1) // cfg["nprint"]]
            assert abs(r[2] - x) < 1e-10 and abs(r[5] - p) < 1e-10, (s, r[2], x, r[5], p)
    # continuum solution of x'' = -x - 0.1 sin(0.9 t): agrees to O(dt^2)
    t = obs[:, 0]
    xc = 2 * np.cos(t) + (0.09 / 0.19) * np.sin(t) - (0.1 / 0.19) * np.sin(0.9 * t)
    assert np.max(np.abs(obs[:, 2] - xc)) < 5e-4
    # squeezed packet breathes: var = 0.25 cos^2 t + sin^2 t, to O(dt^2)
    var = obs[:, 8] - obs[:, 2] ** 2
    assert np.max(np.abs(var - (0.25 * np.cos(t) ** 2 + np.sin(t) ** 2))) < 5e-4
    # norm conservation to round-off over 1000 steps
    assert np.max(np.abs(obs[:, 1] - obs[0, 1])) < 1e-13


def test_laser_trap_2d_follows_verlet_map_per_axis():
    cfg = W.config_2d_laser_trap(n=128)
    pb = dict(cfg["problem"], xmin=[-10.0, -10.0], L=[20.0, 20.0])
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    nt, npr = 500, 50
    psi, obs = O.run(pb, terms, psi0, nt, npr)
    dt = pb["dt"]
    fx = lambda t: 0.05 * math.exp(-((t - 10.0) / 4.0) ** 2) * math.sin(0.5 * t + W.HALF_PI)
    fy = lambda t: 0.0
    st = [(1.0, fx), (4.0, fy)]
    xs = [[obs[0, 2 + d], obs[0, 5 + d]] for d in range(2)]
    for s in range(nt):
        for d in range(2):
            xs[d] = list(verlet_vkv(xs[d][0], xs[d][1], 1.0, st[d][0], st[d][1], (s * dt, (s + 1) * dt), dt))
        if (s + 1) % npr == 0:
            r = obs[(s + 1) // npr]
            for d in range(2):
                assert abs(r[2 + d] - xs[d][0]) < 1e-10 and abs(r[5 + d] - xs[d][1]) < 1e-10


def test_separable_2d_equals_product_of_1d_runs():
    cfg = W.config_2d_laser_trap(n=128)
    pb = dict(cfg["problem"], xmin=[-10.0, -12.0], L=[20.0, 24.0])
    terms = cfg["terms"]
    init = cfg["init"]
    psi2 = O.propagate(pb, terms, O.gaussian(pb, **init), 200)
    rows = []
    for d in range(2):
        p1 = {"ndim": 1, "n": [pb["n"][d]], "xmin": [pb["xmin"][d]], "L": [pb["L"][d]], "mass": 1.0,
              "hbar": 1.0, "dt": pb["dt"], "t0": 0.0, "order": "vkv"}
        t1 = []
        for tm in terms:
            if tm["a"][d] != 0.0:
                t1.append(dict(tm, a=[tm["a"][d]]))
        g = O.gaussian(p1, [init["x0"][d]], [init["p0"][d]], [init["sigma"][d]])
        rows.append(O.propagate(p1, t1, g, 200))
    assert rel_l2(psi2, np.outer(rows[0], rows[1])) < 1e-13


# --------------------------------------------------------------------------- invariants
def test_time_reversibility_vkv():
    cfg = W.config_1d_driven_trap()
    pb = cfg["problem"]
    psi0 = O.gaussian(pb, **cfg["init"])
    n = 300
    psi = O.propagate(pb, cfg["terms"], psi0, n)
    back = dict(pb, dt=-pb["dt"], t0=n * pb["dt"])
    psi_b = O.propagate(back, cfg["terms"], psi, n)
    assert rel_l2(psi_b, psi0) < 1e-12


def barrier_1d(order="vkv", dt=0.01, n=512):
    pb = {"ndim": 1, "n": [n], "xmin": [-30.0], "L": [60.0], "mass": 1.0, "hbar": 1.0, "dt": dt,
          "t0": 0.0, "order": order}
    terms = W.config_3d_barrier()["terms"]
    terms = [dict(terms[0], a=[1.0])]
    return pb, terms, {"x0": [-3.0], "p0": [2.0], "sigma": [1.5]}


@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_second_order_convergence_in_dt(order):
    T = 0.8
    pb, terms, init = barrier_1d(order)
    ref_dt = 0.8 / 1024
    psi0 = O.gaussian(pb, **init)
    ref = O.propagate(dict(pb, dt=ref_dt), terms, psi0, 1024)
    errs = []
    for k in (20, 40, 80):
        errs.append(rel_l2(O.propagate(dict(pb, dt=T / k), terms, psi0, k), ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3, errs
    assert errs[0] > 1e-7  # the barrier really acts


def test_kvk_and_vkv_agree_to_second_order():
    diffs = []
    for k in (40, 80):
        out = []
        for order in ("vkv", "kvk"):
            pb, terms, init = barrier_1d(order, dt=0.8 / k)
            out.append(O.propagate(pb, terms, O.gaussian(pb, **init), k))
        diffs.append(rel_l2(out[0], out[1]))
    assert 3.6 < diffs[0] / diffs[1] < 4.4


def test_energy_static_potential_bounded_no_drift():
    pb, terms, init = barrier_1d("vkv", dt=0.005)
    terms = [dict(terms[0], coef={"A0": 1.5})]
    psi0 = O.gaussian(pb, **init)
    psi, obs = O.run(pb, terms, psi0, 800, 20)
    e = obs[:, 11]
    assert np.max(np.abs(e - e[0])) < 1e-3
    half = len(e) // 2
    # no secular drift: the second half stays as close to E(0) as the first
    assert np.max(np.abs(e[half:] - e[0])) < 2 * np.max(np.abs(e[:half] - e[0])) + 1e-6
    assert np.max(np.abs(obs[:, 1] - 1.0)) < 1e-12


def test_nprint_rules():
    cfg = W.config_1d_driven_trap(n=64)
    pb = dict(cfg["problem"], xmin=[-8.0], L=[16.0])
    psi0 = O.gaussian(pb, **cfg["init"])
    with pytest.raises(ValueError):
        O.run(pb, cfg["terms"], psi0, 5, 6)
    psi, obs = O.run(pb, cfg["terms"], psi0, 7, 3)
    assert obs.shape[0] == 3 and list(obs[:, 15]) == [0.0, 3.0, 6.0]
    assert rel_l2(psi, O.propagate(pb, cfg["terms"], psi0, 7)) == 0.0


def test_potential_terms_pointwise():
    pb = {"ndim": 3, "n": [4, 4, 4], "xmin": [-1.0, -2.0, -3.0], "L": [4.0, 8.0, 12.0], "mass": 1.0,
          "hbar": 1.0, "dt": 0.1, "t0": 0.0}
    terms = [
        {"shape": "quad", "a": [1.0, 2.0, 3.0], "c0": [0.5, 0.0, 0.0], "v": [0.1, 0, 0],
         "coef": {"A0": 0.5, "A": 0.2, "omega": 1.5, "phi": 0.3}},
        {"shape": "gauss", "a": [1.0, 0.0, 2.0], "c0": [0.0, 0.0, 1.0], "coef": {"A0": 2.0}},
        {"shape": "linear", "a": [0.3, 0.0, -0.2],
         "coef": {"A": 1.0, "omega": 2.0, "env": "gauss", "t0": 1.0, "tau": 0.5}},
        {"shape": "morse", "a": [0.4, 1.2, 1.0], "c0": [0.0, 1.5, 0.0],
         "coef": {"A": 1.0, "omega": 0.0, "phi": W.HALF_PI, "env": "sin2", "t0": 0.0, "tau": 4.0}},
        {"shape": "const", "coef": {"A0": -0.25}},
    ]
    t = 1.3
    V = O.potential_grid(pb, terms, t)
    x = np.meshgrid(grid(pb, 0), grid(pb, 1), grid(pb, 2), indexing="ij")
    f1 = 0.5 + 0.2 * math.sin(1.5 * t + 0.3)
    ref = f1 * 0.5 * ((x[0] - 0.5 - 0.1 * t) ** 2 + 2 * x[1] ** 2 + 3 * x[2] ** 2)
    ref += 2.0 * np.exp(-(x[0] ** 2) - ((x[2] - 1.0) / 2.0) ** 2)
    ref += math.exp(-((t - 1.0) / 0.5) ** 2) * math.sin(2 * t) * (0.3 * x[0] - 0.2 * x[2])
    ref += math.sin(math.pi * t / 4.0) ** 2 * math.sin(W.HALF_PI) * 0.4 * (1 - np.exp(-1.2 * (x[1] - 1.5))) ** 2
    ref += -0.25
    assert np.max(np.abs(V - ref) / np.maximum(1.0, np.abs(ref))) < 1e-14


# --------------------------------------------------------------------------- the paper's printed values
def test_paul_trap_printed_widths_are_the_secular_ground_state():
    """Sec. 4.2 prints the trap and the packet widths. The widths are those of the harmonic
    ground state of the lowest-order secular motion, sigma = sqrt(2 hbar/(m w)) in the packet
    convention exp(-x^2/sigma^2). Evaluating the oracle's energy of that packet in the
    secular oscillator gives hbar w/2 up to the 4 printed digits."""
    with open(os.path.join(GOLDEN, "paul_trap_e2.json")) as f:
        g = json.load(f)
    e = W.E_CHARGE_SI
    d2 = g["r0"] ** 2 + 2 * g["z0_over_r0"] ** 2 * g["r0"] ** 2
    Om = 2 * math.pi * g["Omega_over_2pi"]
    qx = 2 * e * g["V0"] / (g["mass"] * d2 * Om ** 2)
    wx = Om / 2 * qx / math.sqrt(2)
    hbar = W.HBAR_SI
    assert abs(math.sqrt(2 * hbar / (g["mass"] * wx)) / g["sigma_x"] - 1) < 1e-3
    assert abs(math.sqrt(2 * hbar / (g["mass"] * 2 * wx)) / g["sigma_z"] - 1) < 1e-3
    # oracle energy of the printed packet in the secular oscillator (SI units)
    n = 256
    pb = {"ndim": 1, "n": [n], "xmin": [-6e-7], "L": [1.2e-6], "mass": g["mass"], "hbar": hbar,
          "dt": 1e-9, "t0": 0.0}
    terms = [{"shape": "quad", "a": [g["mass"] * wx * wx], "coef": {"A0": 1.0}}]
    rec = O.observe(pb, terms, O.gaussian(pb, [0.0], [0.0], [g["sigma_x"]]))
    assert abs(rec[11] / (hbar * wx / 2) - 1) < 1e-5
    assert abs(rec[1] - 1.0) < 1e-12


def test_paul_trap_3d_moments_follow_verlet_map():
    """Sec. 4.2 run on a reduced grid: the quadratic, time-periodic trap gives the exact
    discrete Verlet map for (<x_d>, <p_d>) in SI units."""
    cfg = W.config_paul_trap(n=64)
    pb = dict(cfg["problem"], xmin=[-3.5e-7] * 3, L=[7e-7] * 3)
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    nt, npr = 40, 10
    psi, obs = O.run(pb, terms, psi0, nt, npr)
    tm = terms[0]
    coef = lambda t: tm["coef"]["A0"] + tm["coef"]["A"] * math.sin(tm["coef"]["omega"] * t + tm["coef"]["phi"])
    m, dt = pb["mass"], pb["dt"]
    for d in range(3):
        x, p = obs[0, 2 + d], obs[0, 5 + d]
        for s in range(nt):
            k0, k1 = coef(s * dt) * tm["a"][d], coef((s + 1) * dt) * tm["a"][d]
            p = p - k0 * x * dt / 2
            x = x + p * dt / m
            p = p - k1 * x * dt / 2
            if (s + 1) % npr == 0:
                r = obs[(s + 1) // npr]
                assert abs(r[2 + d] - x) < 1e-12 * abs(x) and abs(r[5 + d] - p) < 1e-12 * 1e-27
    assert np.max(np.abs(obs[:, 1] - 1.0)) < 1e-12


# --------------------------------------------------------------------------- static grid potential
# Sec. 3.2.3: the user potential() gives V at every grid point; a static grid is that
# function evaluated once and added to the analytic terms.
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_constant_grid_potential_is_a_global_phase(order):
    # V = c everywhere: exact solution = free evolution times exp(-i c t / hbar)
    c, hbar, m = 0.37, 0.8, 1.3
    pb = {"ndim": 1, "n": [1024], "xmin": [-20.0], "L": [40.0], "mass": m, "hbar": hbar,
          "dt": 0.01, "t0": 0.0, "order": order}
    psi0 = O.gaussian(pb, [-5.0], [2.0], [1.0])
    psi = O.propagate(dict(pb, vgrid=np.full(1024, c)), [], psi0, 100)
    x = grid(pb, 0)
    ref = free_gaussian_1d(x, 1.0, -5.0, 2.0, 1.0, m, hbar) * np.exp(-1j * c * 1.0 / hbar)
    assert rel_l2(psi, ref) < 1e-12


def test_harmonic_grid_potential_ground_state_3d():
    # V(x) = sum_d w_d^2 x_d^2 / 2 given as a grid: the anisotropic ground state has
    # E = hbar sum w_d / 2 and <x_d^2> = sigma_d^2 / 4, and stays stationary
    w = [1.0, 2.0, 0.5]
    pb = {"ndim": 3, "n": [32, 32, 32], "xmin": [-8.0, -6.0, -12.0], "L": [16.0, 12.0, 24.0],
          "mass": 1.0, "hbar": 1.0, "dt": 0.01, "t0": 0.0, "order": "vkv"}
    X = np.meshgrid(*[grid(pb, d) for d in range(3)], indexing="ij")
    V = sum(0.5 * w[d] ** 2 * X[d] ** 2 for d in range(3))
    pg = dict(pb, vgrid=V)
    sg = [math.sqrt(2.0 / ww) for ww in w]
    psi0 = O.gaussian(pb, [0.0] * 3, [0.0] * 3, sg)
    rec = O.observe(pg, [], psi0)
    assert abs(rec[11] - sum(w) / 2) < 1e-11
    assert abs(rec[13] - sum(w) / 4) < 1e-11
    psi, obs = O.run(pg, [], psi0, 40, 20)
    assert np.max(np.abs(np.abs(psi) ** 2 - np.abs(psi0) ** 2)) < 1e-4
    assert np.max(np.abs(obs[:, 11] - sum(w) / 2)) < 1e-4


def test_grid_adds_to_the_terms():
    # the grid and the terms sum: half a trap as a term plus half as a grid equals the trap
    pb = {"ndim": 2, "n": [32, 64], "xmin": [-6.0, -8.0], "L": [12.0, 16.0], "mass": 1.0, "hbar": 1.0,
          "dt": 0.02, "t0": 0.3, "order": "kvk"}
    full = [{"shape": "quad", "a": [1.0, 0.5], "coef": {"A0": 1.0}},
            {"shape": "linear", "a": [0.3, 0.0], "coef": {"A": 1.0, "omega": 1.1}}]
    half = [{"shape": "quad", "a": [1.0, 0.5], "coef": {"A0": 0.5}}, full[1]]
    X = np.meshgrid(grid(pb, 0), grid(pb, 1), indexing="ij")
    V = 0.25 * (1.0 * X[0] ** 2 + 0.5 * X[1] ** 2)
    psi0 = W.random_state((32, 64), seed=2)
    a = O.propagate(pb, full, psi0, 15)
    b = O.propagate(dict(pb, vgrid=V), half, psi0, 15)
    assert rel_l2(b, a) < 1e-13


# --------------------------------------------------------------------------- Morse (Sec. 4.1)
def test_morse_eigenstates_energy_and_stationarity():
    # the CO Morse potential of Sec. 4.1 on its grid: the closed-form bound states
    # (Morse 1929) have E_v = hbar w (v + 1/2) - (hbar w (v + 1/2))^2 / 4D, and the ground
    # state only turns its phase, e^{-i E_0 t / hbar}
    cfg = W.config_1d_co_morse()
    pb, terms = cfg["problem"], cfg["terms"]
    M = W.CO_MORSE
    dx = pb["L"][0] / pb["n"][0]
    states = [W.morse_eigenstate(pb, v, M["D"], M["a"], M["xe"], W.CO_MASS) for v in range(3)]
    for psi, e in states:
        rec = O.observe(pb, [terms[0]], psi)
        assert abs(rec[1] - 1.0) < 1e-13
        assert abs(rec[11] - e) < 1e-12 * e
    phi0, e0 = states[0]
    psi = O.propagate(pb, [terms[0]], phi0, 2000)
    ov = np.vdot(phi0, psi) * dx
    assert abs(abs(ov) - 1.0) < 1e-12
    assert abs(ov - np.exp(-1j * e0 * 2000 * pb["dt"])) < 1e-6
