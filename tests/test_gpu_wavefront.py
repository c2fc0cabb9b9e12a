"""The synthetic wavefront frame driver: graph replay serves exactly the same
queries as eager launches, the shrinking per-bounce batches follow the
Bernoulli(0.7) survival, and training runs once per frame."""
import math

import numpy as np
import pytest

import synth
from gpu_helpers import make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3, synth.FP16, synth.FP32_TC])
def test_graph_replay_matches_eager(precision):
    import paper_2504_04315_gb300 as npm
    w = synth.TINY
    P, T, frames = 1 << 16, 1 << 12, 3
    stats = {}
    for graph in (False, True):
        m = make_model(w, synth.random_params(w, 61), P, precision=precision)
        with npm.Wavefront(m, P, bounces=8, survival=0.7, train_batch=T, seed=5,
                           use_graph=graph, max_frames=16) as wf:
            stats[graph] = wf.run(frames)
            params = m.get_params()
        stats[graph]["params"] = params
        m.check_device_status()
        m.close()
    a, b = stats[False], stats[True]
    assert a["queries"] == b["queries"]
    expect = frames * P * (1 - 0.7 ** 8) / 0.3
    assert abs(a["queries"] - expect) < 0.01 * expect
    assert math.isfinite(a["last_loss"]) and abs(a["last_loss"] - b["last_loss"]) <= 1e-4 * abs(a["last_loss"])
    assert b["bounce_p99_ms"] >= b["bounce_p50_ms"] > 0 and b["train_ms_mean"] > 0
    # The per-bounce breakdown: live paths per bounce add up to the queries
    # served, shrink bounce by bounce, and the frame's parts fit in its time.
    for st in (a, b):
        assert abs(sum(st["bounce_queries"]) * frames - st["queries"]) < 1e-6 * st["queries"]
        assert st["bounce_queries"][0] == P
        assert all(x > y for x, y in zip(st["bounce_queries"], st["bounce_queries"][1:]))
        assert all(t > 0 for t in st["bounce_query_ms"])
        assert abs(sum(st["bounce_query_ms"]) - st["query_ms_mean"]) < 1e-6 + 1e-6 * st["query_ms_mean"]
        parts = st["query_ms_mean"] + st["advance_ms_mean"] + st["train_ms_mean"]
        assert 0 < parts <= st["frame_ms_mean"] * 1.001
    # Same training trajectory up to the summation order of gradient atomics.
    assert (np.abs(a["params"] - b["params"]) < 1e-5).mean() > 0.999
