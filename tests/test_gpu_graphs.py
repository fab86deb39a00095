"""CUDA-graph replay of repeated step calls on a handle with its own stream: bitwise the
same as direct launches, across chunk lengths, a resumed step index, and after the
potential or the schedule changes (which drop the captured graphs)."""
import numpy as np
import pytest

from paper_1306_3247_gb300 import wavepacket as WPK
from paper_1306_3247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "3d": W.config_3d_barrier(n=32),
    "2d": W.config_2d_laser_trap(n=128),
    "1d": W.config_1d_driven_trap(n=1024),
}


def run(cfg, prec, graphs, plan, extra=None):
    stream = torch.cuda.Stream()
    with WPK.Propagator(cfg["problem"], cfg["terms"], prec, stream=stream.cuda_stream) as P:
        if not graphs:
            P.set_graphs(False)
        P.init_gaussian(**cfg["init"])
        for i, m in enumerate(plan):
            if extra and i in extra:
                extra[i](P)
            P.step(m)
        torch.cuda.synchronize()
        return P.get_state(), P.step_index


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_graph_replay_equals_direct(case, prec):
    cfg = CASES[case]
    plan = [5, 5, 5, 3, 5, 3, 3, 7]
    a, sa = run(cfg, prec, True, plan)
    b, sb = run(cfg, prec, False, plan)
    assert sa == sb == sum(plan)
    assert np.array_equal(a, b)


def test_graphs_dropped_when_the_potential_or_schedule_changes():
    cfg = CASES["3d"]
    new_terms = [{"shape": "quad", "a": [0.2, 0.2, 0.2], "coef": {"A0": 1.0}}]
    extra = {3: lambda P: P.set_potential(new_terms),
             5: lambda P: P.set_schedule(tile_log=10, ept=8, max_radix_log=3, fixed=0)}
    plan = [4, 4, 4, 4, 4, 4, 4]
    a, _ = run(cfg, "c128", True, plan, extra)
    b, _ = run(cfg, "c128", False, plan, extra)
    assert np.array_equal(a, b)


def test_graphs_need_a_stream():
    cfg = CASES["1d"]
    with WPK.Propagator(cfg["problem"], cfg["terms"], "c128") as P:
        with pytest.raises(WPK.WavepacketError) as e:
            P.set_graphs(True)
        assert e.value.status == WPK.WP_EINVAL
