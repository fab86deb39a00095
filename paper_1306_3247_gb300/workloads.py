"""Seeded synthetic workloads for the split-operator step.

This module holds only input descriptions and seeded random draws: grids,
potential-term parameters, Gaussian packet parameters, batched-instance and
request-stream recipes. It contains none of the method's arithmetic (no FFT, no
phase factors, no potential evaluation). Both the CUDA path and the CPU oracle
read their inputs from here and evaluate them with their own code.

Problem dictionary schema:
  ndim         1, 2 or 3 (1-D along x, 2-D in the xy plane)
  n            grid points per axis, powers of two
  xmin, L      first grid point and period per axis (dx = L/n, half-open box)
  mass, hbar   particle mass and hbar (atomic units: hbar = 1)
  dt, t0       time step and initial time; t_n = t0 + n dt
  order        "vkv" (potential half-steps around a full kinetic step) or
               "kvk" (the paper's order: kinetic half-steps around a
               mid-point potential step)

Potential term schema, V(x,t) = sum over terms of f(t) * shape(x,t):
  shape  "const" 1
         "quad"   0.5 * sum_d a_d (x_d - c_d(t))^2
         "linear" sum_d a_d (x_d - c_d(t))
         "gauss"  exp(-sum_{d: a_d > 0} (x_d - c_d(t))^2 / a_d^2)
         "morse"  a_0 (1 - exp(-a_1 (x_k - c_k(t))))^2 along axis k = a_2
  a, c0, v  per-axis parameters; centre c_d(t) = c0_d + v_d t
  coef   {"A0", "A", "omega", "phi", "env", "t0", "tau"}:
         f(t) = A0 + A env(t) sin(omega t + phi),
         env "none" -> 1, "gauss" -> exp(-(t - t0)^2 / tau^2),
         "sin2" -> sin^2(pi t / tau) on t0 <= t <= t0 + tau, else 0.

Initial state: {"x0", "p0", "sigma"} of the normalised Gaussian packet
  prod_d exp(i p0_d (x_d - x0_d)/hbar) exp(-(x_d - x0_d)^2 / sigma_d^2).
"""
import math

import numpy as np

HALF_PI = math.pi / 2


def _problem(ndim, n, xmin, L, dt, mass=1.0, hbar=1.0, t0=0.0, order="vkv"):
    return {"ndim": ndim, "n": list(n), "xmin": list(xmin), "L": list(L), "mass": mass,
            "hbar": hbar, "dt": dt, "t0": t0, "order": order}


def config_1d_driven_trap(n=1024, order="vkv"):
    """1-D, N=1024 on [-20, 20), V = x^2/2 + 0.1 sin(0.9 t) x, packet sigma=1 at x0=2,
    dt=0.01, 1000 steps, observables every 10 steps."""
    pb = _problem(1, [n], [-20.0], [40.0], 0.01, order=order)
    terms = [
        {"shape": "quad", "a": [1.0], "coef": {"A0": 1.0}},
        {"shape": "linear", "a": [1.0], "coef": {"A": 0.1, "omega": 0.9}},
    ]
    init = {"x0": [2.0], "p0": [0.0], "sigma": [1.0]}
    return {"name": "1d_driven_trap_N%d" % n, "problem": pb, "terms": terms, "init": init,
            "nt": 1000, "nprint": 10}


def config_2d_laser_trap(n=1024, order="vkv"):
    """2-D n x n on [-40, 40)^2, V = (x^2 + 4 y^2)/2 + E0 exp(-(t-t0)^2/tau^2) cos(wL t) x
    (E0=0.05, wL=0.5, t0=10, tau=4), packet sigma=(1, 0.7), p0=(1, 0) at the origin,
    dt=0.005, 500 steps."""
    pb = _problem(2, [n, n], [-40.0, -40.0], [80.0, 80.0], 0.005, order=order)
    terms = [
        {"shape": "quad", "a": [1.0, 4.0], "coef": {"A0": 1.0}},
        {"shape": "linear", "a": [1.0, 0.0],
         "coef": {"A": 0.05, "omega": 0.5, "phi": HALF_PI, "env": "gauss", "t0": 10.0, "tau": 4.0}},
    ]
    init = {"x0": [0.0, 0.0], "p0": [1.0, 0.0], "sigma": [1.0, 0.7]}
    return {"name": "2d_laser_trap_%dx%d" % (n, n), "problem": pb, "terms": terms, "init": init,
            "nt": 500, "nprint": 50}


def config_3d_barrier(n=256, order="vkv"):
    """3-D n^3 on [-30, 30)^3: packet sigma=1.5, p0=(2,0,0) at (-3,0,0) hitting a spherical
    Gaussian barrier 1.5 (1 + 0.3 sin 2t) exp(-|r|^2) at the origin, dt=0.002, 200 steps."""
    pb = _problem(3, [n, n, n], [-30.0] * 3, [60.0] * 3, 0.002, order=order)
    terms = [{"shape": "gauss", "a": [1.0, 1.0, 1.0], "coef": {"A0": 1.5, "A": 0.45, "omega": 2.0}}]
    init = {"x0": [-3.0, 0.0, 0.0], "p0": [2.0, 0.0, 0.0], "sigma": [1.5, 1.5, 1.5]}
    return {"name": "3d_barrier_%d^3" % n, "problem": pb, "terms": terms, "init": init,
            "nt": 200, "nprint": 20}


# Constants for the ion-trap example (Sec. 4.2, Tab. 2, CODATA 2010).
HBAR_SI = 1.054571726e-34
E_CHARGE_SI = 1.602176565e-19


def config_paul_trap(n=512, nt=18500):
    """The paper's Ba+ Paul-trap run (Sec. 4.2), SI units: V = e (U0 + V0 cos Omega t)
    (x^2 + y^2 - 2 z^2) / (2 d^2), d^2 = r0^2 + 2 z0^2, grid n^3 on [-1e-6, 1e-6] m."""
    m = 2.28997005e-25
    V0, U0 = 200.0, 0.0
    Om = 2 * math.pi * 18e6
    r0 = 1.6e-3
    z0 = r0 / math.sqrt(2.0)
    d2 = r0 * r0 + 2 * z0 * z0
    kappa = E_CHARGE_SI / d2  # V = kappa (U0 + V0 cos) * 0.5 * (x^2 + y^2 - 2 z^2)
    # paper-style closed grid [-1e-6, 1e-6] with n points: L = n (xmax - xmin)/(n - 1)
    xmin, xmax = -1e-6, 1e-6
    L = n * (xmax - xmin) / (n - 1)
    pb = _problem(3, [n] * 3, [xmin] * 3, [L] * 3, 2e-9, mass=m, hbar=HBAR_SI)
    terms = [{"shape": "quad", "a": [kappa, kappa, -2 * kappa],
              "coef": {"A0": U0, "A": V0, "omega": Om, "phi": HALF_PI}}]
    # a = (kappa, kappa, -2 kappa), f(t) = U0 + V0 cos(Omega t): V = f(t) * 0.5 sum a_d x_d^2
    init = {"x0": [2e-8, 1e-8, 2e-8], "p0": [1e-27, 0.0, 0.0], "sigma": [7.342e-8, 7.342e-8, 5.192e-8]}
    return {"name": "paul_trap_%d^3" % n, "problem": pb, "terms": terms, "init": init,
            "nt": nt, "nprint": 10}


# The paper's CO example (Sec. 4.1): 12C16O in a Morse potential driven by a resonant
# 1 ps laser pulse through its dipole moment, atomic units.
CO_MASS = 12498.10
CO_MORSE = {"D": 0.4076, "a": 1.230211, "xe": 2.1322214}
CO_DIPOLE = {"mu0": -0.1466, "mu1": -0.948}
CO_PULSE = {"E0": 1.69e-3, "omega": 9.8864e-3, "ti": 0.0, "tf": 41341.37}


def config_1d_co_morse(n=4096, nt=500000, nprint=20000, t0=0.0, order="vkv"):
    """Sec. 4.1: V = D (1 - exp(-a (x - xe)))^2 + (mu0 + mu1 (x - xe)) E0 f(t) cos(omega t),
    f = sin^2(pi t / (tf - ti)) on [ti, tf]; the paper's grid of 4000 points on
    [1.5e-3, 6] becomes 4096 points on the same closed interval (L = n (xmax - xmin)/(n - 1));
    dt = 0.1, 500 000 steps, projections every 20 000. Initial state: the Morse ground state
    (morse_eigenstate)."""
    xmin, xmax = 1.5e-3, 6.0
    L = n * (xmax - xmin) / (n - 1)
    pb = _problem(1, [n], [xmin], [L], 0.1, mass=CO_MASS, t0=t0, order=order)
    M, Dp, P = CO_MORSE, CO_DIPOLE, CO_PULSE
    pulse = {"omega": P["omega"], "phi": HALF_PI, "env": "sin2", "t0": P["ti"], "tau": P["tf"] - P["ti"]}
    terms = [
        {"shape": "morse", "a": [M["D"], M["a"], 0.0], "c0": [M["xe"]], "coef": {"A0": 1.0}},
        {"shape": "linear", "a": [Dp["mu1"]], "c0": [M["xe"]], "coef": dict(pulse, A=P["E0"])},
        {"shape": "const", "coef": dict(pulse, A=Dp["mu0"] * P["E0"])},
    ]
    return {"name": "1d_co_morse_N%d" % n, "problem": pb, "terms": terms, "nt": nt, "nprint": nprint}


def morse_eigenstate(pb, v, D, a, xe, mass, hbar=1.0):
    """Bound state v of D (1 - exp(-a (x - xe)))^2 on the 1-D grid of pb, normalised on the
    grid: the textbook closed form (Morse 1929) with lam = sqrt(2 m D)/(a hbar),
    z = 2 lam exp(-a (x - xe)): psi_v ~ z^(lam - v - 1/2) exp(-z/2) L_v^(2 lam - 2 v - 1)(z),
    energy hbar w (v + 1/2) - (hbar w (v + 1/2))^2 / (4 D), w = a sqrt(2 D / m). Returns
    (psi, energy)."""
    n = int(pb["n"][0])
    x = pb["xmin"][0] + np.arange(n) * (pb["L"][0] / n)
    lam = math.sqrt(2.0 * mass * D) / (a * hbar)
    if not v < lam - 0.5:
        raise ValueError("v beyond the last bound state")
    z = 2.0 * lam * np.exp(-a * (x - xe))
    alpha = 2.0 * lam - 2.0 * v - 1.0
    lag_prev, lag = np.ones_like(z), 1.0 + alpha - z  # generalised Laguerre recurrence
    if v == 0:
        lag = lag_prev
    else:
        for k in range(1, v):
            lag_prev, lag = lag, ((2 * k + 1 + alpha - z) * lag - (k + alpha) * lag_prev) / (k + 1)
    logamp = (lam - v - 0.5) * np.log(z) - 0.5 * z
    with np.errstate(divide="ignore"):
        logamp = logamp + np.log(np.abs(lag))
    psi = np.sign(lag) * np.exp(logamp - logamp.max())
    psi = psi / math.sqrt(float(np.sum(psi * psi)) * pb["L"][0] / n)
    w = a * math.sqrt(2.0 * D / mass)
    e = hbar * w * (v + 0.5) - (hbar * w * (v + 0.5)) ** 2 / (4.0 * D)
    return psi.astype(np.complex128), e


def random_state(shape, seed):
    """Seeded complex normal noise (for transform tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def batched_instances(count=4096, seed=1306):
    """Uneven batch of independent driven-trap propagations: 1-D or 2-D by a fair coin,
    1-D N in {2^8..2^13}, 2-D each axis in {64, 128, 256}, trap frequency w in U[0.5, 2],
    drive amplitude A in U[0, 0.2] at Omega = 0.9 w, centred Gaussian with
    sigma = sqrt(2/w) U[0.7, 1.3], box L = 16 sigma n / 256 clipped to >= 20, dt = 0.005."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        two_d = rng.random() < 0.5
        if two_d:
            n = [int(rng.choice([64, 128, 256])), int(rng.choice([64, 128, 256]))]
        else:
            n = [int(2 ** rng.integers(8, 14))]
        w = float(rng.uniform(0.5, 2.0))
        A = float(rng.uniform(0.0, 0.2))
        sig = math.sqrt(2.0 / w) * float(rng.uniform(0.7, 1.3))
        nd = len(n)
        L = [max(20.0, 16.0 * sig * nn / 256.0) for nn in n]
        pb = _problem(nd, n, [-l / 2 for l in L], L, 0.005)
        terms = [
            {"shape": "quad", "a": [w * w] * nd, "coef": {"A0": 1.0}},
            {"shape": "linear", "a": [1.0] + [0.0] * (nd - 1), "coef": {"A": A, "omega": 0.9 * w}},
        ]
        init = {"x0": [0.0] * nd, "p0": [0.0] * nd, "sigma": [sig] * nd}
        out.append({"name": "inst%d" % i, "problem": pb, "terms": terms, "init": init})
    return out


def request_stream(count=2000, rate=200.0, seed=3247):
    """Poisson stream of propagation requests: dimension uniform over {1,2,3}; 1-D 2^10..2^14,
    2-D 2^8..2^10 per axis, 3-D 2^6..2^8 per axis; 100..2000 steps; driven trap or moving
    barrier plus a weak trap. Returns a list of (arrival_time_s, job dict)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        nd = int(rng.integers(1, 4))
        if nd == 1:
            n = [int(2 ** rng.integers(10, 15))]
        elif nd == 2:
            e = int(2 ** rng.integers(8, 11))
            n = [e, e]
        else:
            e = int(2 ** rng.integers(6, 9))
            n = [e, e, e]
        steps = int(rng.integers(100, 2001))
        L = [40.0] * nd
        pb = _problem(nd, n, [-20.0] * nd, L, 0.005)
        if rng.random() < 0.5:
            w = float(rng.uniform(0.5, 2.0))
            terms = [
                {"shape": "quad", "a": [w * w] * nd, "coef": {"A0": 1.0}},
                {"shape": "linear", "a": [1.0] + [0.0] * (nd - 1),
                 "coef": {"A": float(rng.uniform(0.0, 0.2)), "omega": 0.9 * w}},
            ]
            init = {"x0": [1.0] + [0.0] * (nd - 1), "p0": [0.0] * nd, "sigma": [math.sqrt(2.0 / w)] * nd}
        else:
            h = float(rng.uniform(0.5, 3.0))
            wb = float(rng.uniform(0.5, 1.5))
            vb = float(rng.uniform(-1.0, 1.0))
            terms = [
                {"shape": "quad", "a": [0.01] * nd, "coef": {"A0": 1.0}},
                {"shape": "gauss", "a": [wb] + [0.0] * (nd - 1), "c0": [2.0] + [0.0] * (nd - 1),
                 "v": [vb] + [0.0] * (nd - 1), "coef": {"A0": h}},
            ]
            init = {"x0": [-4.0] + [0.0] * (nd - 1), "p0": [2.0] + [0.0] * (nd - 1), "sigma": [1.0] * nd}
        out.append((t, {"name": "req%d" % i, "problem": pb, "terms": terms, "init": init,
                        "nt": steps, "nprint": steps}))
    return out
