"""Batched instances: every instance's result in the batch equals the result it gives
alone (same kernels' arithmetic, bitwise), and matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def small_mix(count=24, seed=5):
    inst = W.batched_instances(count=count, seed=seed)
    out = []
    for cfg in inst:
        pb = dict(cfg["problem"])
        if pb["ndim"] == 1:
            pb["n"] = [min(pb["n"][0], 2048)]
        out.append(dict(cfg, problem=pb))
    return out


@pytest.mark.parametrize("prec", ["c128", "c64", "c128f"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(prec, use_graph):
    mix = small_mix()
    with WPK.Batch(prec) as B:
        for cfg in mix:
            k = B.add(cfg["problem"], cfg["terms"])
            B.init_gaussian(k, **cfg["init"])
        for _ in range(3):
            B.step(7, use_graph=use_graph)
        got = [B.get_state(k) for k in range(len(mix))]
        assert B.launches > 0
    for k, cfg in enumerate(mix):
        with WPK.Propagator(cfg["problem"], cfg["terms"], prec) as P:
            P.init_gaussian(**cfg["init"])
            for _ in range(3):
                P.step(7)
            alone = P.get_state()
        assert np.array_equal(got[k], alone), (k, cfg["problem"]["n"], rel_l2(got[k], alone))


def test_batch_matches_oracle_c128():
    mix = small_mix(count=8, seed=11)
    with WPK.Batch("c128") as B:
        for cfg in mix:
            k = B.add(cfg["problem"], cfg["terms"])
            B.init_gaussian(k, **cfg["init"])
        B.step(40)
        got = [B.get_state(k) for k in range(len(mix))]
    for k, cfg in enumerate(mix):
        pb, terms = cfg["problem"], cfg["terms"]
        ref = O.propagate(pb, terms, O.gaussian(pb, **cfg["init"]), 40)
        assert rel_l2(got[k], ref) < 1e-11, (k, pb["n"])


def test_batch_kvk_and_mixed_dims():
    mix = small_mix(count=6, seed=2)
    extra = W.config_3d_barrier(n=16)
    with WPK.Batch("c128") as B:
        for cfg in mix:
            pb = dict(cfg["problem"], order="kvk")
            k = B.add(pb, cfg["terms"])
            B.init_gaussian(k, **cfg["init"])
        k3 = B.add(extra["problem"], extra["terms"])
        B.init_gaussian(k3, **extra["init"])
        B.step(9)
        B.step(9)
        got = [B.get_state(k) for k in range(len(mix) + 1)]
    cfgs = [dict(c, problem=dict(c["problem"], order="kvk")) for c in mix] + [extra]
    for k, cfg in enumerate(cfgs):
        pb, terms = cfg["problem"], cfg["terms"]
        ref = O.propagate(pb, terms, O.gaussian(pb, **cfg["init"]), 18)
        assert rel_l2(got[k], ref) < 1e-11, (k, pb["n"])


def test_batch_matches_oracle_c64():
    # the complex64 batch (two-stage kernels for 64-, 128- and 256-point axes, Stockham
    # for the rest) against the oracle, within the form's 2e-4
    mix = small_mix(count=12, seed=13)
    with WPK.Batch("c64") as B:
        for cfg in mix:
            k = B.add(cfg["problem"], cfg["terms"])
            B.init_gaussian(k, **cfg["init"])
        B.step(40)
        got = [B.get_state(k) for k in range(len(mix))]
    for k, cfg in enumerate(mix):
        pb, terms = cfg["problem"], cfg["terms"]
        ref = O.propagate(pb, terms, O.gaussian(pb, **cfg["init"]), 40)
        assert rel_l2(got[k], ref) < 2e-4, (k, pb["n"])
