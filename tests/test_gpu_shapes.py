"""Edge shapes through both paths against the oracle: the widest layers and
most lobes the library takes (NPM_MAX_WIDTH 128, K = 16), 8 and 1 features
per level, an odd level count mixing dense and hashed levels."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import (DIR_TOL_FP32, MARGIN_FP32, PDF_RTOL_FP32, compare_samples, cuda, host,
                         make_model)
from test_gpu_tc import _bf16_stats

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# 3 levels (6^3 and 20^3 dense, 90^3 hashed into 2^16), 8 features, widest
# hidden layers, K = 16.
WIDE = synth.Workload(name="3 levels x 8 feats, MLP 24-128-128-64, K=16", mode=synth.RADIANCE,
                      level_res=[6, 20, 90], feat=8, log2_table=16, widths=[24, 128, 128, 64], K=16,
                      n_query=2048, n_train=2048)
# K = 16 with layers narrow enough for tensor-core training.
LOBES16 = WIDE.with_(name="3 levels x 8 feats, MLP 24-64-64, K=16", widths=[24, 64, 64])
# 8 levels of one feature (5 dense, 3 hashed into 2^17), K = 2.
ONEFEAT = synth.Workload(name="8 levels x 1 feat, MLP 8-16-16-8, K=2", mode=synth.RADIANCE,
                         level_res=[4, 7, 12, 20, 33, 55, 90, 150], feat=1, log2_table=17,
                         widths=[8, 16, 16, 8], K=2, n_query=2048, n_train=2048)
SHAPES = [WIDE, LOBES16, ONEFEAT]


@pytest.fixture(autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@pytest.mark.parametrize("precision", [synth.FP32, synth.FP32_TC], ids=["fp32", "fp32-tc"])
@pytest.mark.parametrize("w", SHAPES, ids=lambda w: w.name[:24])
def test_fp32_sampling_and_indices(w, precision):
    # Both FP32-accuracy paths (CUDA cores; tensor cores with split FP16
    # operands) at the FP32 bars.
    n = 3000
    params = synth.random_params(w, 31)
    pos, u = synth.positions(31, n), synth.sample_uniforms(31, n)
    m = make_model(w, params, n, precision=precision)
    assert np.array_equal(host(m.grid_indices(cuda(pos))), oracle.grid_indices(w, pos))
    d, p, _ = m.query_sample(cuda(pos), cuda(u))
    stats = compare_samples(w, params, pos, u, None, 0.0, host(d), host(p), PDF_RTOL_FP32,
                            DIR_TOL_FP32, MARGIN_FP32)
    print(w.name, stats)


@pytest.mark.parametrize("w", SHAPES, ids=lambda w: w.name[:24])
def test_split_bf16_sampling(w):
    err, *_ = _bf16_stats(w.with_(precision=synth.BF16X3), 4096, 32, precision=synth.BF16X3)
    print(f"{w.name}: pdf err p50 {np.median(err):.2e} p99.9 {np.quantile(err, 0.999):.2e}")
    assert np.quantile(err, 0.999) <= 2e-2


@pytest.mark.parametrize("w,precision,bar", [(LOBES16, synth.FP32, 1e-4), (ONEFEAT, synth.FP32, 1e-4),
                                             (LOBES16, synth.BF16X3, 2e-2),
                                             (ONEFEAT, synth.BF16X3, 2e-2)],
                         ids=["lobes16-fp32", "onefeat-fp32", "lobes16-split", "onefeat-split"])
def test_gradients(w, precision, bar):
    n = 2048
    params = synth.random_params(w, 33)
    b = synth.train_batch_uniform(w, n, seed=33)
    m = make_model(w, params, n, precision=precision)
    dlogv = -(b.radiance.astype(np.float64) / b.pdf) / n
    m.backward(cuda(b.pos), cuda(b.dir), cuda(dlogv))
    m.check_device_status()
    g = m.get_grads()
    _, ref = oracle.train_grad(w, params, b.pos, b.dir, b.radiance, b.pdf)
    ng = sum(synth.grid_sizes(w)) * w.feat
    blocks = [("grid", slice(0, ng))]
    o = ng
    for i in range(len(w.widths) - 1):
        k = w.widths[i] * w.widths[i + 1]
        blocks.append((f"W{i + 1}", slice(o, o + k)))
        o += k
    errs = {name: np.linalg.norm(g[sl] - ref[sl]) / max(np.linalg.norm(ref[sl]), 1e-30)
            for name, sl in blocks}
    print(w.name, precision, errs)
    assert max(errs.values()) <= bar, errs


@pytest.mark.parametrize("precision", [synth.FP32, synth.BF16X3])
def test_training_too_wide_is_refused_cleanly(precision):
    # WIDE's per-tile activations exceed shared memory for both training
    # kernels: the call returns NPM_ERR_UNSUPPORTED without launching, and
    # the handle keeps working.
    from paper_2504_04315_gb300 import NpmError
    n = 256
    params = synth.random_params(WIDE, 34)
    b = synth.train_batch_uniform(WIDE, n, seed=34)
    m = make_model(WIDE, params, n, precision=precision)
    with pytest.raises(NpmError) as ei:
        m.train_step(cuda(b.pos), cuda(b.dir), cuda(b.radiance), cuda(b.pdf))
    assert ei.value.status == 7  # NPM_ERR_UNSUPPORTED
    assert np.array_equal(m.get_params(), params)
    d, p, _ = m.query_sample(cuda(b.pos), cuda(synth.sample_uniforms(34, n)))
    assert np.all(np.isfinite(host(p)))
