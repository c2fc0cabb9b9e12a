"""Moving average of the weights for inference (Sec. 5.3; npm_set_ema):
the average the Adam kernel keeps matches the oracle's, inference evaluates
it, and training is unaffected by it."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import cuda, host, make_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _batch(w, n, seed):
    b = synth.train_batch_uniform(w, n, seed=seed)
    return [cuda(a) if a is not None else None for a in (b.pos, b.dir, b.radiance, b.pdf, b.aux)]


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3, synth.FP32_TC])
def test_ema_tracks_oracle_and_serves_inference(precision):
    w = synth.TINY.with_(precision=precision)
    n, decay, steps = 4096, 0.9, 8
    params = synth.random_params(w, 61)
    m = make_model(w, params, n)
    m.set_ema(decay)
    assert np.array_equal(m.get_ema_params(), params)  # starts at the parameters
    e = params.astype(np.float64)
    tb = _batch(w, n, 61)
    for _ in range(steps):
        m.train_step(tb[0], tb[1], tb[2], tb[3], tb[4])
        oracle.ema(e, m.get_params(), decay)
    got = m.get_ema_params().astype(np.float64)
    assert np.abs(got - e).max() <= 1e-6 * np.abs(e).max() + 1e-9, np.abs(got - e).max()
    assert np.abs(got - m.get_params()).max() > 0  # the average lags the parameters

    # Inference evaluates the average: same outputs as a model whose
    # parameters are the average.
    ref = make_model(w, m.get_ema_params(), n)
    pos, u = cuda(synth.positions(62, n)), cuda(synth.sample_uniforms(62, n))
    d1, p1, _ = m.query_sample(pos, u)
    d2, p2, _ = ref.query_sample(pos, u)
    assert torch.equal(d1, d2) and torch.equal(p1, p2)
    q1 = m.eval_pdf(pos, d1)
    q2 = ref.eval_pdf(pos, d1)
    assert torch.equal(q1, q2)

    # Off again: inference evaluates the parameters.
    m.set_ema(0.0)
    cur = make_model(w, m.get_params(), n)
    d3, p3, _ = m.query_sample(pos, u)
    d4, p4, _ = cur.query_sample(pos, u)
    assert torch.equal(d3, d4) and torch.equal(p3, p4)
    for x in (m, ref, cur):
        x.close()


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3])
def test_training_is_unaffected_by_ema(precision):
    w = synth.TINY.with_(precision=precision)
    n = 4096
    params = synth.random_params(w, 63)
    a, b = make_model(w, params, n), make_model(w, params, n)
    a.set_ema(0.99)
    tb = _batch(w, n, 63)
    for _ in range(5):
        a.train_step(tb[0], tb[1], tb[2], tb[3], tb[4])
        b.train_step(tb[0], tb[1], tb[2], tb[3], tb[4])
    # Same updates; the grid gradients are sums of atomic adds, whose order
    # (and so the last bits) varies from run to run.
    pa, pb = a.get_params(), b.get_params()
    assert np.abs(pa - pb).max() <= 1e-5 * np.abs(pb).max(), np.abs(pa - pb).max()
    a.close()
    b.close()
