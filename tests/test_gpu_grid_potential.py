"""Static grid potentials (the user potential() of Sec. 3.2.3 evaluated on the grid), given
as an array or as CUDA source compiled at run time: parity with the oracle (which adds the
same grid to V), observables, batching, removal and compile errors."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-11, "c128f": 1e-11, "c64": 2e-4}
OBS_TOL = {"c128": 1e-10, "c128f": 1e-10, "c64": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    WPK.load_library()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def coords(pb):
    nd = pb["ndim"]
    ax = [pb["xmin"][d] + np.arange(pb["n"][d]) * pb["L"][d] / pb["n"][d] for d in range(nd)]
    return np.meshgrid(*ax, indexing="ij")


def landscape(pb, seed):
    """A smooth seeded landscape: a few Gaussian wells and bumps plus a weak anharmonic wall."""
    rng = np.random.default_rng(seed)
    X = coords(pb)
    V = np.zeros(X[0].shape)
    for _ in range(4):
        c = [rng.uniform(-2, 2) for _ in X]
        h = rng.uniform(-1.0, 1.5)
        V += h * np.exp(-sum((x - cc) ** 2 for x, cc in zip(X, c)) / rng.uniform(0.5, 2.0))
    V += 0.01 * sum(x ** 4 for x in X)
    return V


def compare_obs(obs, ref, rtol):
    M = WPK.obs_matrix(obs)
    assert np.array_equal(M[:, 15], ref[:, 15])
    scale = np.maximum(np.max(np.abs(ref[:, 1:15]), axis=0), 1.0)
    err = np.max(np.abs(M[:, 1:15] - ref[:, 1:15]), axis=0) / scale
    assert np.all(err < rtol), err


CASES = {
    "3d": ({"ndim": 3, "n": [16, 32, 64], "xmin": [-4.0, -5.0, -6.0], "L": [8.0, 10.0, 12.0], "mass": 1.0,
            "hbar": 1.0, "dt": 0.01, "t0": 0.0},
           [{"shape": "quad", "a": [0.5, 0.5, 0.5], "coef": {"A0": 1.0}},
            {"shape": "gauss", "a": [1.0, 1.0, 1.0], "c0": [0.5, 0.0, 0.0], "coef": {"A0": 0.5, "A": 0.2,
                                                                                   "omega": 2.0}}]),
    "2d_long_axis": ({"ndim": 2, "n": [32, 2048], "xmin": [-6.0, -20.0], "L": [12.0, 40.0], "mass": 1.0,
                      "hbar": 1.0, "dt": 0.005, "t0": 0.0},
                     [{"shape": "linear", "a": [0.2, 0.1], "coef": {"A": 1.0, "omega": 0.9}}]),
    "1d_fixed": ({"ndim": 1, "n": [1024], "xmin": [-20.0], "L": [40.0], "mass": 1.0, "hbar": 1.0, "dt": 0.01,
                  "t0": 0.0},
                 [{"shape": "linear", "a": [1.0], "coef": {"A": 0.1, "omega": 0.9}}]),
    "1d_short": ({"ndim": 1, "n": [64], "xmin": [-8.0], "L": [16.0], "mass": 1.0, "hbar": 1.0, "dt": 0.01,
                  "t0": 0.0}, []),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["c128", "c64", "c128f"])
@pytest.mark.parametrize("order", ["vkv", "kvk"])
def test_grid_potential_matches_oracle(case, prec, order):
    pb, terms = CASES[case]
    pb = dict(pb, order=order)
    V = landscape(pb, seed=len(case))
    nd = pb["ndim"]
    init = {"x0": [0.3] * nd, "p0": [0.5] * nd, "sigma": [1.0] * nd}
    psi0 = O.gaussian(pb, **init)
    nt, npr = 40, 10
    ref, ref_obs = O.run(dict(pb, vgrid=V), terms, psi0, nt, npr)
    with WPK.Propagator(pb, terms, prec, autocorr=True) as P:
        P.set_potential_grid(V)
        P.set_state(psi0)
        obs = P.run(nt, npr)
        psi = P.get_state()
    assert rel_l2(psi, ref) < TOL[prec]
    compare_obs(obs, ref_obs, OBS_TOL[prec])


def test_grid_removed_equals_no_grid():
    pb, terms = CASES["3d"]
    psi0 = W.random_state((16, 32, 64), seed=4)
    with WPK.Propagator(pb, terms, "c128") as P:
        P.set_potential_grid(landscape(pb, 1))
        P.set_potential_grid(None)
        P.set_state(psi0)
        P.step(10)
        a = P.get_state()
    with WPK.Propagator(pb, terms, "c128") as Q:
        Q.set_state(psi0)
        Q.step(10)
        b = Q.get_state()
    assert np.array_equal(a, b)


def test_grid_from_device_tensor():
    torch = pytest.importorskip("torch")
    pb, terms = CASES["3d"]
    V = landscape(pb, 2)
    psi0 = W.random_state((16, 32, 64), seed=5)
    ref = O.propagate(dict(pb, vgrid=V), terms, psi0, 8)
    with WPK.Propagator(pb, terms, "c128") as P:
        P.set_potential_grid(torch.from_numpy(V).cuda())
        P.set_state(psi0)
        P.step(8)
        assert rel_l2(P.get_state(), ref) < 1e-11


SRC_HARMONIC = """
__device__ double wp_user_potential(double x, double y, double z) {
  return 0.5 * (1.0 * x * x + 4.0 * y * y) + 0.25 * z;
}
"""


def test_source_potential_equals_terms():
    pb = {"ndim": 3, "n": [32, 32, 16], "xmin": [-6.0, -6.0, -4.0], "L": [12.0, 12.0, 8.0], "mass": 1.0,
          "hbar": 1.0, "dt": 0.01, "t0": 0.0}
    terms = [{"shape": "quad", "a": [1.0, 4.0, 0.0], "coef": {"A0": 1.0}},
             {"shape": "linear", "a": [0.0, 0.0, 0.25], "coef": {"A0": 1.0}}]
    psi0 = W.random_state((32, 32, 16), seed=6)
    X = coords(pb)
    V = 0.5 * (X[0] ** 2 + 4.0 * X[1] ** 2) + 0.25 * X[2]
    ref = O.propagate(dict(pb, vgrid=V), [], psi0, 20)
    with WPK.Propagator(pb, [], "c128") as P:
        P.set_potential_source(SRC_HARMONIC)
        P.set_state(psi0)
        P.step(20)
        a = P.get_state()
    with WPK.Propagator(pb, terms, "c128") as Q:
        Q.set_state(psi0)
        Q.step(20)
        b = Q.get_state()
    assert rel_l2(a, ref) < 1e-11
    assert rel_l2(a, b) < 1e-11


def test_source_compile_error_is_reported():
    pb, terms = CASES["1d_short"]
    with WPK.Propagator(pb, terms, "c128") as P:
        with pytest.raises(WPK.WavepacketError) as e:
            P.set_potential_source("__device__ double wp_user_potential(double x, double y, double z) { return q; }")
        assert e.value.status == WPK.WP_EINVAL
        assert "compile" in str(e.value)


def test_batched_instances_with_grids_equal_alone():
    inst = W.batched_instances(count=16)
    pick = [c for c in inst if c["problem"]["ndim"] == 1][:2] + [c for c in inst if c["problem"]["ndim"] == 2][:2]
    alone = []
    for c in pick:
        with WPK.Propagator(c["problem"], c["terms"], "c64") as P:
            P.set_potential_grid(landscape(c["problem"], 9))
            P.init_gaussian(**c["init"])
            P.step(12)
            alone.append(P.get_state())
    B = WPK.Batch("c64")
    try:
        for c in pick:
            k = B.add(c["problem"], c["terms"])
            shape = tuple(c["problem"]["n"][: c["problem"]["ndim"]])
            V = np.ascontiguousarray(landscape(c["problem"], 9))
            assert V.shape == shape
            WPK.wp_set_potential_grid(B.handle(k), V.ctypes.data, False)
            B.init_gaussian(k, **c["init"])
        B.step(12, use_graph=True)
        for k in range(len(pick)):
            assert np.array_equal(B.get_state(k), alone[k])
    finally:
        B.close()
