"""Pass schedules and the autotuner: every schedule computes the same step (parity with
the FP64 oracle within the form's tolerance), the autotuner restores the state and step
index it timed on, caches its choice by shape, and later handles of that shape (alone
or batched) run with it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def candidates(ndim):
    out = [{"tile_log": 11, "ept": 8, "max_radix_log": 3, "fixed": 1}]
    if ndim > 1:
        for tl in (10, 11, 12):
            for e in (8, 16):
                for r in (2, 3):
                    out.append({"tile_log": tl, "ept": e, "max_radix_log": r, "fixed": 0})
    else:
        for e in (8, 16):
            for r in (2, 3):
                out.append({"tile_log": 11, "ept": e, "max_radix_log": r, "fixed": 0})
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(autouse=True)
def _clean_cache():
    WPK.load_library()
    WPK.wp_autotune_cache_clear()
    yield
    WPK.wp_autotune_cache_clear()


PROBLEMS = {
    "3d": ({"ndim": 3, "n": [16, 32, 64], "xmin": [-4.0, -5.0, -6.0], "L": [8.0, 10.0, 12.0], "mass": 1.0,
            "hbar": 1.0, "dt": 0.01, "t0": 0.2},
           [{"shape": "quad", "a": [1.0, 0.5, 2.0], "coef": {"A0": 1.0}},
            {"shape": "gauss", "a": [1.0, 1.5, 1.0], "c0": [0.2, 0.0, -0.1], "v": [0.1, 0.0, 0.0],
             "coef": {"A0": 1.5, "A": 0.3, "omega": 2.0}}]),
    "2d": ({"ndim": 2, "n": [64, 4096], "xmin": [-6.0, -20.0], "L": [12.0, 40.0], "mass": 0.8, "hbar": 1.0,
            "dt": 0.005, "t0": 0.0},
           [{"shape": "quad", "a": [1.0, 0.3], "coef": {"A0": 1.0}},
            {"shape": "linear", "a": [0.4, 0.0], "coef": {"A": 1.0, "omega": 0.9}}]),
    "1d": ({"ndim": 1, "n": [4096], "xmin": [-20.0], "L": [40.0], "mass": 1.0, "hbar": 1.0, "dt": 0.01,
            "t0": 0.0},
           [{"shape": "quad", "a": [1.0], "coef": {"A0": 1.0}},
            {"shape": "linear", "a": [1.0], "coef": {"A": 0.1, "omega": 0.9}},
            {"shape": "gauss", "a": [0.7], "c0": [1.0], "coef": {"A0": 0.5, "A": 0.2, "omega": 1.3}}]),
}


@pytest.mark.parametrize("name", ["3d", "2d", "1d"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_every_schedule_matches_oracle(name, prec):
    pb, terms = PROBLEMS[name]
    shape = tuple(pb["n"][: pb["ndim"]])
    psi0 = W.random_state(shape, seed=11)
    nsteps = 12
    ref = O.propagate(pb, terms, psi0, nsteps)
    tol = 1e-11 if prec == "c128" else 2e-4
    ran = 0
    for sc in candidates(pb["ndim"]):
        with WPK.Propagator(pb, terms, prec) as P:
            try:
                P.set_schedule(**sc)
            except WPK.WavepacketError as e:
                assert e.status == WPK.WP_EUNSUPPORTED
                continue
            assert P.schedule == sc
            P.set_state(psi0)
            P.step(5)
            P.step(nsteps - 5)
            err = rel_l2(P.get_state(), ref)
            assert err < tol, (sc, err)
            ran += 1
    assert ran >= (5 if pb["ndim"] > 1 else 3)


def test_schedule_field_range_is_checked():
    pb, terms = PROBLEMS["3d"]
    with WPK.Propagator(pb, terms, "c128") as P:
        before = P.schedule
        for bad in ({"tile_log": 9}, {"ept": 4}, {"max_radix_log": 4}, {"fixed": 2}):
            with pytest.raises(WPK.WavepacketError) as e:
                P.set_schedule(**bad)
            assert e.value.status == WPK.WP_EINVAL
        assert P.schedule == before


@pytest.mark.parametrize("name", ["3d", "1d"])
def test_autotune_restores_state_and_caches(name):
    pb, terms = PROBLEMS[name]
    shape = tuple(pb["n"][: pb["ndim"]])
    psi0 = W.random_state(shape, seed=12)
    with WPK.Propagator(pb, terms, "c128") as P:
        P.set_state(psi0)
        P.step(3)
        before = P.get_state()
        sched, ms, ncand = P.autotune(steps=2)
        assert ncand >= 3 and ms > 0.0
        assert sched in candidates(pb["ndim"])
        assert P.schedule == sched
        assert P.step_index == 3
        assert np.array_equal(P.get_state(), before)
        P.step(9)
        ref = O.propagate(pb, terms, psi0, 12)
        assert rel_l2(P.get_state(), ref) < 1e-11
    assert WPK.wp_autotune_cache_size() == 1
    with WPK.Propagator(pb, terms, "c128") as Q:
        assert Q.schedule == sched
    with WPK.Propagator(pb, terms, "c64") as R:  # another key
        assert R.schedule == candidates(pb["ndim"])[0]
    WPK.wp_autotune_cache_clear()
    with WPK.Propagator(pb, terms, "c128") as S:
        assert S.schedule == candidates(pb["ndim"])[0]


def test_batched_1d_instances_follow_their_schedule():
    inst = [c for c in W.batched_instances(count=64) if c["problem"]["ndim"] == 1][:6]
    sched = {"tile_log": 11, "ept": 16, "max_radix_log": 2, "fixed": 0}
    alone = []
    for c in inst:
        with WPK.Propagator(c["problem"], c["terms"], "c64") as P:
            P.set_schedule(**sched)
            P.init_gaussian(**c["init"])
            P.step(20)
            alone.append(P.get_state())
    B = WPK.Batch("c64")
    try:
        for c in inst:
            k = B.add(c["problem"], c["terms"])
            WPK.wp_set_schedule(B.handle(k), sched)
            B.init_gaussian(k, **c["init"])
        B.step(20, use_graph=True)
        for k in range(len(inst)):
            assert np.array_equal(B.get_state(k), alone[k])
    finally:
        B.close()


@pytest.mark.parametrize("prec,tol", [("c128", 1e-14), ("c128f", 1e-13), ("c64", 1e-7)])
def test_initial_gaussian_3d_matches_oracle(prec, tol):
    pb, terms = PROBLEMS["3d"]
    init = {"x0": [0.3, -0.4, 0.5], "p0": [1.0, -0.5, 2.0], "sigma": [0.9, 1.3, 1.1]}
    ref = O.gaussian(pb, **init)
    with WPK.Propagator(pb, terms, prec) as P:
        P.init_gaussian(**init)
        assert rel_l2(P.get_state(), ref) < tol
