"""User observables (Sec. 3.2.5): a grid operator's expectation value and a per-record
host callback that sees the record's state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    WPK.load_library()


def coords(pb):
    nd = pb["ndim"]
    ax = [pb["xmin"][d] + np.arange(pb["n"][d]) * pb["L"][d] / pb["n"][d] for d in range(nd)]
    return np.meshgrid(*ax, indexing="ij")


@pytest.mark.parametrize("prec,tol", [("c128", 1e-13), ("c128f", 1e-12), ("c64", 1e-6)])
@pytest.mark.parametrize("shape", [(1024,), (32, 64), (16, 16, 32)])
def test_expect_grid_matches_direct_sum(prec, tol, shape):
    nd = len(shape)
    pb = {"ndim": nd, "n": list(shape), "xmin": [-4.0] * nd, "L": [8.0] * nd, "mass": 1.0, "hbar": 1.0,
          "dt": 0.01, "t0": 0.0}
    X = coords(pb)
    A = np.cos(X[0]) + sum(0.1 * x * x for x in X)
    psi = W.random_state(shape, seed=7)
    dv = np.prod([8.0 / n for n in shape])
    ref = float(np.sum(A * np.abs(psi) ** 2) * dv)
    with WPK.Propagator(pb, [], prec) as P:
        P.set_state(psi)
        got = P.expect_grid(A)
        assert abs(got - ref) <= tol * abs(ref)
        assert P.expect_grid(A) == got  # fixed reduction order


def test_expect_grid_of_x_equals_record():
    cfg = W.config_3d_barrier(n=32)
    pb, terms = cfg["problem"], cfg["terms"]
    with WPK.Propagator(pb, terms, "c128") as P:
        P.init_gaussian(**cfg["init"])
        P.step(10)
        rec = P.observe()
        X = coords(pb)
        for d in range(3):
            assert abs(P.expect_grid(X[d]) - rec["x%d" % d]) < 1e-12


@pytest.mark.parametrize("nt,nprint", [(60, 20), (50, 20)])
def test_run_callback_records_equal_run(nt, nprint):
    cfg = W.config_2d_laser_trap(n=128)
    pb = dict(cfg["problem"], xmin=[-10.0, -10.0], L=[20.0, 20.0])
    terms = cfg["terms"]
    psi0 = O.gaussian(pb, **cfg["init"])
    with WPK.Propagator(pb, terms, "c128") as P:
        P.set_state(psi0)
        ref = WPK.obs_matrix(P.run(nt, nprint))
        ref_state = P.get_state()
    seen, norms = [], []
    X = coords(pb)
    with WPK.Propagator(pb, terms, "c128") as Q:
        Q.set_state(psi0)

        def fn(prop, rec):
            seen.append(rec)
            norms.append(prop.expect_grid(np.ones_like(X[0])))
            assert prop.step_index == int(rec["step"])
            return False

        n = Q.run_with_callback(nt, nprint, fn)
        state = Q.get_state()
    M = WPK.obs_matrix(np.array(seen))
    assert n == len(seen) == ref.shape[0] == 1 + nt // nprint
    assert np.array_equal(M[:, 15], ref[:, 15])
    assert np.allclose(M, ref, rtol=1e-12, atol=1e-14)
    assert np.allclose(np.sqrt(norms), M[:, 1], rtol=1e-12)
    assert np.abs(state - ref_state).max() < 1e-13


def test_run_callback_stops_early():
    pb = {"ndim": 1, "n": [256], "xmin": [-10.0], "L": [20.0], "mass": 1.0, "hbar": 1.0, "dt": 0.01, "t0": 0.0}
    with WPK.Propagator(pb, [{"shape": "quad", "a": [1.0], "coef": {"A0": 1.0}}], "c128") as P:
        P.init_gaussian([1.0], [0.0], [1.0])
        n = P.run_with_callback(100, 10, lambda prop, rec: int(rec["step"]) >= 30)
        assert n == 4
        assert P.step_index == 30
