"""The paper's CO example (Sec. 4.1): a Morse oscillator driven through its dipole by a
resonant 1 ps sin^2-envelope pulse, started in the closed-form ground state. Parity with
the oracle on a mid-pulse segment, and the paper's full 500 000-step run with the
projections on the first five vibrational states as user observables (Sec. 3.2.5),
compared between the native FP64 and the float-float forms."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M = W.CO_MORSE


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    WPK.load_library()


@pytest.mark.parametrize("prec,tol", [("c128", 1e-11), ("c128f", 1e-11), ("c64", 2e-4)])
def test_mid_pulse_segment_matches_oracle(prec, tol):
    t_mid = 0.5 * (W.CO_PULSE["tf"] - W.CO_PULSE["ti"])
    cfg = W.config_1d_co_morse(t0=t_mid)
    pb, terms = cfg["problem"], cfg["terms"]
    phi0, _ = W.morse_eigenstate(pb, 0, M["D"], M["a"], M["xe"], W.CO_MASS)
    ref, ref_obs = O.run(pb, terms, phi0, 2000, 500)
    with WPK.Propagator(pb, terms, prec) as P:
        P.set_state(phi0)
        obs = WPK.obs_matrix(P.run(2000, 500))
        psi = P.get_state()
    assert rel_l2(psi, ref) < tol
    scale = np.maximum(np.max(np.abs(ref_obs[:, 1:14]), axis=0), 1e-3)
    assert np.all(np.max(np.abs(obs[:, 1:14] - ref_obs[:, 1:14]), axis=0) / scale < max(tol, 1e-10) * 10)


def projections_run(prec, nt, nprint):
    cfg = W.config_1d_co_morse(nt=nt, nprint=nprint)
    pb, terms = cfg["problem"], cfg["terms"]
    dx = pb["L"][0] / pb["n"][0]
    phis = [W.morse_eigenstate(pb, v, M["D"], M["a"], M["xe"], W.CO_MASS)[0] for v in range(5)]
    rows = []
    with WPK.Propagator(pb, terms, prec) as P:
        P.set_state(phis[0])

        def observe(prop, rec):
            psi = prop.get_state()
            rows.append([float(rec["t"]), float(rec["norm"])] + [abs(np.vdot(f, psi) * dx) ** 2 for f in phis])
            return False

        n = P.run_with_callback(nt, nprint, observe)
    assert n == 1 + nt // nprint
    return np.array(rows)


def test_paper_run_projections_native_vs_float_float():
    nt, nprint = 500000, 20000
    a = projections_run("c128", nt, nprint)
    b = projections_run("c128f", nt, nprint)
    assert np.max(np.abs(a[:, 1] - 1.0)) < 1e-10          # norm
    assert np.max(np.abs(a[:, 2:] - b[:, 2:])) < 1e-9      # both forms agree
    assert np.all(a[:, 2:].sum(axis=1) <= a[:, 1] ** 2 + 1e-12)  # at most the norm^2
    assert a[0, 2] > 1.0 - 1e-12                           # starts in v = 0
    # the resonant pulse moves population out of v = 0 into v = 1 (and a little beyond);
    # after the pulse (t >= tf) the populations stay fixed
    assert a[-1, 3] > 0.05 and a[-1, 2] < 0.95
    after = a[a[:, 0] >= W.CO_PULSE["tf"]]
    assert np.max(np.ptp(after[:, 2:], axis=0)) < 1e-6
    print("t, norm, P_0..P_4:\n" + "\n".join(" ".join("%.6g" % x for x in r) for r in a))
